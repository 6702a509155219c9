// sg_guess.cu -- initial guesses: extrapolation (Sec. 3) and right-hand-side
// projection (Sec. 2, Algorithms 1 and 2).
//
// Extrapolation keeps a ring of the last s solutions; the guess is one
// streaming pass x0 = sum_i beta_i x_{ring(i)} (Eq. ExtrapExpn) with beta
// from Eq. LSQRCoeffs (or Eq. CPQRCoeffs, zero terms skipped).
//
// Projection keeps B~ (orthonormal right-hand-side basis) and X~ (A X~ = B~)
// in s physical column slots, logical column j = scale_j * slot_j.  Storing
// the new column unnormalised with scale 1/||b~|| folds the normalisation
// (paper kernel rhsUpdateSpace) into the last Gram-Schmidt sweep.  The
// update (Algorithm 2 after the solve) is four launches:
//   sem_apply : t = A x_k
//   upd1      : [d = M: drop column 1 of R, d-1 Givens rotations of the column
//               pairs of B~ and X~ in one register-carried sweep] + c1 = B~^T t,
//               ||t||^2                          (rhsQRUpdate + rhsProject)
//   upd2      : t -= B~ c1, c2 = B~^T t          (rhsReconstruct + rhsProject)
//   upd3      : t -= B~ c2 -> slot d of B~; x~ = x_k - X~ (c1 + c2) -> slot d
//               of X~; ||t||^2; accept if ||t|| > eps ||A x_k||, d++
// The x~ updates of both CGS passes are merged into one (X~ is not modified
// in between).  All control (d, R, Givens parameters, the eps test) runs in
// the last CTA of each sweep, so nothing synchronises with the host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sg_sem_launch.cuh"

namespace sgb {
int lsq_beta(int M, int m, double* beta);
int sparse_beta(int M, int m, double* beta);
}

namespace {
constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr int NV = SG_SMAX + 1;   // dots + one norm per reduction
}

struct ProjState {
  int d, accepted, rotated, pad;
  double R[SG_SMAX * SG_SMAX];   // row-major, R[i*SMAX + j]
  double scale[SG_SMAX];
  double c1[SG_SMAX], c2[SG_SMAX], alpha[SG_SMAX];
  double nrm0sq, nrmsq;
  unsigned int counter[4];
};

struct sg_guess_s {
  int method, s, m, dtype, nsl;   // nsl: ring slots (EXTRAP family)
  int64_t n;
  double eps_rel;
  sg_op_t op;
  unsigned char* ws;
  size_t off_state, off_partials, off_a, off_b, off_t, slot_bytes;
  int blocks;
  int count, next;                // ring bookkeeping (host mirror, deterministic)
  double beta_tab[SG_SMAX + 1][SG_SMAX];
};

template <typename T> struct VecT;
template <> struct VecT<double> { using V = double2; static constexpr int W = 2; };
template <> struct VecT<float> { using V = float4; static constexpr int W = 4; };

// lane accessors; w is a compile-time constant after unrolling, so the
// vectors stay in registers
__device__ __forceinline__ double& vel(double2& v, int w) { return w == 0 ? v.x : v.y; }
__device__ __forceinline__ float& vel(float4& v, int w) {
  return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}
__device__ __forceinline__ double vel(const double2& v, int w) { return w == 0 ? v.x : v.y; }
__device__ __forceinline__ float vel(const float4& v, int w) {
  return w == 0 ? v.x : (w == 1 ? v.y : (w == 2 ? v.z : v.w));
}
template <typename V> __device__ __forceinline__ V vzero() { V v; for (int w = 0; w < (int)(sizeof(V) / sizeof(v.x)); ++w) vel(v, w) = 0; return v; }

// Column counts are compile-time template arguments: GB300's FP64 pipe is narrow
// enough that predicated-off multiply-adds of a fixed 16-column loop would cost
// as much as live ones.  The host dispatches the extrapolation kernel on its
// term count; the projection kernels read d on the device and switch (block-
// uniformly) to the body instantiated for that d.
#define SG_COLS_DISPATCH(d, CALL)                                                         \
  switch (d) {                                                                            \
    case 0: CALL(0); break;   case 1: CALL(1); break;   case 2: CALL(2); break;           \
    case 3: CALL(3); break;   case 4: CALL(4); break;   case 5: CALL(5); break;           \
    case 6: CALL(6); break;   case 7: CALL(7); break;   case 8: CALL(8); break;           \
    case 9: CALL(9); break;   case 10: CALL(10); break; case 11: CALL(11); break;         \
    case 12: CALL(12); break; case 13: CALL(13); break; case 14: CALL(14); break;         \
    case 15: CALL(15); break; case 16: CALL(16); break; default: break;                   \
  }

// The same for the projection kernels, instantiated only up to DMAX columns
// (DMAX = the history size s rounded up to 4, 8 or 16; d never exceeds s), so a
// kernel's registers are sized for the largest column count it can meet.
#define SG_COLS_CASE(DMAX, k, CALL) case k: if constexpr ((k) <= (DMAX)) { CALL(k); } break;
#define SG_COLS_DISPATCH_UPTO(DMAX, d, CALL)                                              \
  switch (d) {                                                                            \
    SG_COLS_CASE(DMAX, 0, CALL) SG_COLS_CASE(DMAX, 1, CALL) SG_COLS_CASE(DMAX, 2, CALL)    \
    SG_COLS_CASE(DMAX, 3, CALL) SG_COLS_CASE(DMAX, 4, CALL) SG_COLS_CASE(DMAX, 5, CALL)    \
    SG_COLS_CASE(DMAX, 6, CALL) SG_COLS_CASE(DMAX, 7, CALL) SG_COLS_CASE(DMAX, 8, CALL)    \
    SG_COLS_CASE(DMAX, 9, CALL) SG_COLS_CASE(DMAX, 10, CALL) SG_COLS_CASE(DMAX, 11, CALL)  \
    SG_COLS_CASE(DMAX, 12, CALL) SG_COLS_CASE(DMAX, 13, CALL) SG_COLS_CASE(DMAX, 14, CALL) \
    SG_COLS_CASE(DMAX, 15, CALL) SG_COLS_CASE(DMAX, 16, CALL) default: break;              \
  }

// ---------------------------------------------------------------- extrapolation
template <typename T>
struct ExtrapArgs {
  const T* src[SG_SMAX];
  double beta[SG_SMAX];
  int k;
};

// FP64 grid-stride sweeps are software pipelined: the loads of the thread's
// next element are issued before the FP64 work on this one, so memory and the
// FP64 pipe (2 operations per clock per SM on GB300) overlap instead of
// alternating.  Such sweeps run 2 CTAs of 256 per SM (PIPE_CTAS_PER_SM), ~9
// elements per thread at 1.44M nodes, with two register sets of columns.
constexpr int kPipeMaxCols = 9;   // columns a pipelined sweep holds per register set
constexpr int PIPE_CTAS_PER_SM = 2;

template <typename T> constexpr bool pipelined(int cols) { return sizeof(T) == 8 && cols <= kPipeMaxCols; }

// The thread's grid-stride elements i < nv: load(i, buf) fills NB vectors,
// body(i, buf) consumes them; the next element's loads are issued before
// this element's body runs (its stores come after them in program order).
template <typename V, int NB, typename LoadF, typename BodyF>
__device__ __forceinline__ void pipe_loop(int nv, LoadF load, BodyF body) {
  const int stride = gridDim.x * blockDim.x;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  V cur[NB];
  if (i < nv) load(i, cur);
  for (; i < nv; i += stride) {
    V nxt[NB];
    const int in = i + stride;
    if (in < nv) load(in, nxt);
    body(i, cur);
#pragma unroll
    for (int k = 0; k < NB; ++k) cur[k] = nxt[k];
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_extrap(T* out, const ExtrapArgs<T> a, int n) {
  using V = typename VecT<T>::V;
  constexpr int W = VecT<T>::W;
  T b[K];
#pragma unroll
  for (int j = 0; j < K; ++j) b[j] = (T)a.beta[j];
  const int nv = n / W;
  const int stride = gridDim.x * blockDim.x;
  int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (pipelined<T>(K)) {
    V va[K];
    if (i0 < nv) {
#pragma unroll
      for (int j = 0; j < K; ++j) va[j] = reinterpret_cast<const V*>(a.src[j])[i0];
    }
    for (int i = i0; i < nv; i += stride) {
      const int inext = i + stride;
      V vb[K];
      if (inext < nv) {
#pragma unroll
        for (int j = 0; j < K; ++j) vb[j] = reinterpret_cast<const V*>(a.src[j])[inext];
      }
      V acc;
#pragma unroll
      for (int w = 0; w < W; ++w) vel(acc, w) = b[0] * vel(va[0], w);
#pragma unroll
      for (int j = 1; j < K; ++j)
#pragma unroll
        for (int w = 0; w < W; ++w) vel(acc, w) = fma(b[j], vel(va[j], w), vel(acc, w));
      reinterpret_cast<V*>(out)[i] = acc;
#pragma unroll
      for (int j = 0; j < K; ++j) va[j] = vb[j];
    }
    i0 = nv;   // the vector loop is done
  }
  for (int i = i0; i < nv; i += stride) {
    V v[K];
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = reinterpret_cast<const V*>(a.src[j])[i];   // all loads in flight
    V acc;
#pragma unroll
    for (int w = 0; w < W; ++w) vel(acc, w) = b[0] * vel(v[0], w);
#pragma unroll
    for (int j = 1; j < K; ++j)
#pragma unroll
      for (int w = 0; w < W; ++w) vel(acc, w) += b[j] * vel(v[j], w);
    reinterpret_cast<V*>(out)[i] = acc;
  }
  for (int i = nv * W + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    T acc = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) acc += b[j] * a.src[j][i];
    out[i] = acc;
  }
}

// ---------------------------------------------------------------- projection kernels
template <typename T>
struct ProjArgs {
  T* B;              // slot 0 of B~ (slot j at B + j*stride)
  T* X;              // slot 0 of X~
  T* t;              // temporary right-hand side (b~ during the update)
  const T* v;        // form: b;  upd3: x_k
  T* out;            // form: x0
  size_t stride;     // elements between slots
  int n, M, classic;
  int energy;        // inner products in the A-inner product (A-orthonormal X~)
  double eps_rel;
  ProjState* st;
  double* partials;
};

template <typename T>
__device__ __forceinline__ const typename VecT<T>::V* colv(const T* base, size_t stride, int j) {
  return reinterpret_cast<const typename VecT<T>::V*>(base + (size_t)j * stride);
}

#define SG_NZ(D) ((D) > 0 ? (D) : 1)

// v[j] += slot_j . y for j < D (plain dots; the caller applies column scales)
template <typename T, int D, int N>
__device__ __forceinline__ void dots_body(const T* base, size_t stride, const T* y, int n, double (&v)[N]) {
  using V = typename VecT<T>::V;
  constexpr int W = VecT<T>::W;
  T acc[SG_NZ(D)];
#pragma unroll
  for (int j = 0; j < D; ++j) acc[j] = 0;
  const int nv = n / W, stride_i = gridDim.x * blockDim.x;
  if constexpr (pipelined<T>(D + 1)) {
    pipe_loop<V, D + 1>(nv,
      [&](int i, V (&buf)[D + 1]) {
        buf[D] = reinterpret_cast<const V*>(y)[i];
#pragma unroll
        for (int j = 0; j < D; ++j) buf[j] = colv(base, stride, j)[i];
      },
      [&](int, V (&buf)[D + 1]) {
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
          for (int w = 0; w < W; ++w) acc[j] = fma(vel(buf[j], w), vel(buf[D], w), acc[j]);
      });
  } else {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride_i) {
      const V yv = reinterpret_cast<const V*>(y)[i];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const V cv = colv(base, stride, j)[i];
#pragma unroll
        for (int w = 0; w < W; ++w) acc[j] += vel(cv, w) * vel(yv, w);
      }
    }
  }
  for (int i = nv * W + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride_i) {
#pragma unroll
    for (int j = 0; j < D; ++j) acc[j] += base[(size_t)j * stride + i] * y[i];
  }
#pragma unroll
  for (int j = 0; j < D; ++j) v[j] = (double)acc[j];
}

// form, pass 1: alpha_j = scale_j * (slot_j . b), j < d
// The reductions carry DMAX values (+ a norm) rather than SG_SMAX: the block
// sum costs about as many additions per thread as the padded value count.
template <typename T, int DMAX>
__global__ void __launch_bounds__(256) k_proj_dots(const ProjArgs<T> a) {
  __shared__ double sred[32 * DMAX];
  const int d = a.st->d;
  double v[DMAX], tot[DMAX];
#pragma unroll
  for (int j = 0; j < DMAX; ++j) v[j] = 0.0;
  const T* partner = a.energy ? a.X : a.B;   // energy: alpha = X~^T b = (X~, A^{-1} b)_A
#define SG_CALL(D) dots_body<T, D>(partner, a.stride, a.v, a.n, v)
  SG_COLS_DISPATCH_UPTO(DMAX, d, SG_CALL)
#undef SG_CALL
  if (grid_reduce_last<DMAX>(v, a.partials, &a.st->counter[0], sred, tot)) {
    if (threadIdx.x == 0)
      for (int j = 0; j < d; ++j) a.st->alpha[j] = a.st->scale[j] * tot[j];
  }
}

// out = sum_j c_j slot_j, j < D
template <typename T, int D>
__device__ __forceinline__ void lincomb_body(const T* base, size_t stride, const T (&c)[SG_SMAX], T* out, int n) {
  using V = typename VecT<T>::V;
  constexpr int W = VecT<T>::W;
  const int nv = n / W, stride_i = gridDim.x * blockDim.x;
  if constexpr (D > 0 && pipelined<T>(D)) {
    pipe_loop<V, D>(nv,
      [&](int i, V (&buf)[D]) {
#pragma unroll
        for (int j = 0; j < D; ++j) buf[j] = colv(base, stride, j)[i];
      },
      [&](int i, V (&buf)[D]) {
        V acc = vzero<V>();
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
          for (int w = 0; w < W; ++w) vel(acc, w) = fma(c[j], vel(buf[j], w), vel(acc, w));
        reinterpret_cast<V*>(out)[i] = acc;
      });
  } else {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride_i) {
      V xs[SG_NZ(D)];
#pragma unroll
      for (int j = 0; j < D; ++j) xs[j] = colv(base, stride, j)[i];
      V acc = vzero<V>();
#pragma unroll
      for (int j = 0; j < D; ++j)
#pragma unroll
        for (int w = 0; w < W; ++w) vel(acc, w) += c[j] * vel(xs[j], w);
      reinterpret_cast<V*>(out)[i] = acc;
    }
  }
  for (int i = nv * W + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride_i) {
    T acc = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) acc += c[j] * base[(size_t)j * stride + i];
    out[i] = acc;
  }
}

// form, pass 2: x0 = sum_j alpha_j scale_j slot_j of X~ (x0 untouched if d = 0)
template <typename T, int DMAX>
__global__ void __launch_bounds__(256) k_proj_lincomb(const ProjArgs<T> a) {
  const int d = a.st->d;
  if (d == 0) return;
  T c[SG_SMAX];
#pragma unroll
  for (int j = 0; j < SG_SMAX; ++j) c[j] = (j < d) ? (T)(a.st->alpha[j] * a.st->scale[j]) : (T)0;
#define SG_CALL(D) lincomb_body<T, D>(a.X, a.stride, c, a.out, a.n)
  SG_COLS_DISPATCH_UPTO(DMAX, d, SG_CALL)
#undef SG_CALL
}

// One Givens sweep over a column set (App. A: the column shared by successive
// rotations stays in registers): D rotations, new columns 0..D-1 written back,
// dots of the new B~ columns with t accumulated when DOTS.
//
// The rotations are normally applied in factored ("fast Givens", Gentleman
// 1973) form on unscaled columns: a rotation of the pair (C, N) with column
// scales (sc, sn) -- true columns sc C, sn N -- writes new = X + k1 Y and
// carries X' = Y + k2 X (one multiply-add each, X/Y = C/N or N/C as gr.swap
// says), the factor taken out going into the column scales; thread 0 of the
// block computes k1, k2, swap and the scales from c and s (k_proj_upd1).  That
// is half the FP64 operations of applying c and s directly.  The scales drift
// by the factors taken out, so once one leaves a safe range the sweep runs in
// the plain form instead, new = q0 C + q1 N, carry = q2 C + q3 N on a carry
// that starts as sc0 C, which leaves every new column with scale 1.
template <typename T>
struct GivensCoef {
  T k1[SG_SMAX], k2[SG_SMAX];   // factored form
  int swap[SG_SMAX];
  T q[4][SG_SMAX];              // plain form
  T sc0;
};

template <typename T, int D, bool DOTS, bool FAST>
__device__ __forceinline__ void givens_sweep(T* base, size_t stride, const T* t, int n, const GivensCoef<T>& gr,
                                             T (&acc)[SG_NZ(D)]) {
  using V = typename VecT<T>::V;
  constexpr int W = VecT<T>::W;
  const int nv = n / W, stride_i = gridDim.x * blockDim.x;
  // one element: the D + 1 columns (and t) are loaded before the first new
  // column is stored -- loads after a store to the same array would wait for
  // it, a load latency per rotation
  auto rotate = [&](int i, V (&cols)[D + 2]) {
    const V tv = cols[D + 1];
    V carry = cols[0];
    if (!FAST) {
#pragma unroll
      for (int w = 0; w < W; ++w) vel(carry, w) *= gr.sc0;
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const V nx = cols[j + 1];
      V o;
      if (FAST) {
        // coefficients re-read from shared memory on every element: held in
        // registers across the loop they would cost 3 per rotation
        const bool sw = reinterpret_cast<const volatile int*>(gr.swap)[j] != 0;
        const T k1 = reinterpret_cast<const volatile T*>(gr.k1)[j];
        const T k2 = reinterpret_cast<const volatile T*>(gr.k2)[j];
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const T x = sw ? vel(nx, w) : vel(carry, w);
          const T y = sw ? vel(carry, w) : vel(nx, w);
          vel(o, w) = fma(k1, y, x);
          vel(carry, w) = fma(k2, x, y);
        }
      } else {
        const volatile T* q = &gr.q[0][0];
        const T q0 = q[j], q1 = q[SG_SMAX + j], q2 = q[2 * SG_SMAX + j], q3 = q[3 * SG_SMAX + j];
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const T cv = vel(carry, w), nv_ = vel(nx, w);
          vel(o, w) = q0 * cv + q1 * nv_;
          vel(carry, w) = q2 * cv + q3 * nv_;
        }
      }
      if (DOTS) {
#pragma unroll
        for (int w = 0; w < W; ++w) acc[j] += vel(o, w) * vel(tv, w);
      }
      reinterpret_cast<V*>(base + (size_t)j * stride)[i] = o;
    }
  };
  auto load = [&](int i, V (&cols)[D + 2]) {
    if (DOTS) cols[D + 1] = reinterpret_cast<const V*>(t)[i];
#pragma unroll
    for (int j = 0; j <= D; ++j) cols[j] = colv(base, stride, j)[i];
  };
  if constexpr (pipelined<T>(D + 2)) {
    pipe_loop<V, D + 2>(nv, load, rotate);
  } else {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride_i) {
      V cols[D + 2];
      load(i, cols);
      rotate(i, cols);
    }
  }
  for (int i = nv * W + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride_i) {
    const T tt = DOTS ? t[i] : (T)0;
    T carry = base[i];
    if (!FAST) carry *= gr.sc0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const T nx = base[(size_t)(j + 1) * stride + i];
      T o;
      if (FAST) {
        const bool sw = gr.swap[j] != 0;
        const T x = sw ? nx : carry, y = sw ? carry : nx;
        o = fma(gr.k1[j], y, x);
        carry = fma(gr.k2[j], x, y);
      } else {
        o = gr.q[0][j] * carry + gr.q[1][j] * nx;
        carry = gr.q[2][j] * carry + gr.q[3][j] * nx;
      }
      if (DOTS) acc[j] += o * tt;
      base[(size_t)j * stride + i] = o;
    }
  }
}

template <typename T, int D, bool EN, int N>
__device__ __forceinline__ void givens_body(const ProjArgs<T>& a, const GivensCoef<T>& gr, bool fast,
                                            double (&v)[N]) {
  T acc[SG_NZ(D)];
#pragma unroll
  for (int j = 0; j < D; ++j) acc[j] = 0;
  // CGS pass-1 dots with the rotated columns: B~ (Euclidean) or X~ (energy)
  if (fast) {
    givens_sweep<T, D, !EN, true>(a.B, a.stride, a.t, a.n, gr, acc);
    givens_sweep<T, D, EN, true>(a.X, a.stride, a.t, a.n, gr, acc);
  } else {
    givens_sweep<T, D, !EN, false>(a.B, a.stride, a.t, a.n, gr, acc);
    givens_sweep<T, D, EN, false>(a.X, a.stride, a.t, a.n, gr, acc);
  }
#pragma unroll
  for (int j = 0; j < D; ++j) v[j] = (double)acc[j];
}

// u . t (u = t: ||t||^2)
template <typename T>
__device__ __forceinline__ T vdot(const T* u, const T* t, int n) {
  using V = typename VecT<T>::V;
  constexpr int W = VecT<T>::W;
  T nn = 0;
  const int nv = n / W, stride_i = gridDim.x * blockDim.x;
  if constexpr (pipelined<T>(2)) {
    pipe_loop<V, 2>(nv,
      [&](int i, V (&buf)[2]) { buf[0] = reinterpret_cast<const V*>(t)[i]; buf[1] = reinterpret_cast<const V*>(u)[i]; },
      [&](int, V (&buf)[2]) {
#pragma unroll
        for (int w = 0; w < W; ++w) nn = fma(vel(buf[1], w), vel(buf[0], w), nn);
      });
  } else {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride_i) {
      const V tv = reinterpret_cast<const V*>(t)[i];
      const V uv = reinterpret_cast<const V*>(u)[i];
#pragma unroll
      for (int w = 0; w < W; ++w) nn += vel(uv, w) * vel(tv, w);
    }
  }
  for (int i = nv * W + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride_i) nn += u[i] * t[i];
  return nn;
}

// update sweep 1: optional Givens downdate (Algorithm 2, d = M) or classic
// restart (Algorithm 1, d = 0 or d >= M), then c1 = B~^T t and ||t||^2
// (energy: c1 = X~^T t = (X~, x_k)_A and ||x_k||_A^2 = x_k . t).
template <typename T, bool EN, int DMAX>
// FP32: 3 CTAs per SM (85 registers): the rotation sweep is bound by the loads
// in flight, and the extra CTA beats the few spills it costs.  FP64: 2 CTAs
// per SM with the pipelined sweep's two register sets of columns.
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? PIPE_CTAS_PER_SM : 3) k_proj_upd1(const ProjArgs<T> a) {
  constexpr int RV = DMAX + 1;           // dots, then ||t||^2 at [DMAX]
  __shared__ double sred[32 * RV];
  __shared__ double sR[SG_SMAX * SG_SMAX];
  __shared__ GivensCoef<T> gr;
  __shared__ double s_sc[SG_SMAX];      // column scales before the downdate
  __shared__ double s_scale[SG_SMAX];   // column scales after the downdate
  __shared__ double s_cr[SG_SMAX], s_sr[SG_SMAX];
  const int tid = threadIdx.x;
  // every thread reads the same history size (the state changes only in the
  // last block, after all blocks have passed this point)
  const ProjState* st = a.st;
  int d = st->d;
  int rot = 0;
  if (a.classic) {
    if (d >= a.M) d = 0;   // hard restart: the new vector starts a fresh space
  } else if (d == a.M && d > 1) {
    rot = 1;
  } else if (d == a.M && d == 1) {
    d = 0;   // dropping the only column leaves an empty space
  }
  bool fast = true;
  if (rot) {
    // R <- R(:, 2:d): a d x (d-1) upper Hessenberg matrix
    for (int k = tid; k < d * (d - 1); k += blockDim.x) {
      const int i = k / (d - 1), j = k - i * (d - 1);
      sR[i * SG_SMAX + j] = st->R[i * SG_SMAX + j + 1];
    }
    if (tid < d) s_sc[tid] = st->scale[tid];
    __syncthreads();
    // factored form while every scale stays within 2^-e..2^e (stored values
    // then stay far from overflow and underflow in T)
    const double lim = sizeof(T) == 8 ? 0x1p300 : 0x1p40;
    for (int j = 0; j < d; ++j) {
      const double m = fabs(s_sc[j]);
      if (!(m < lim && m > 1.0 / lim)) fast = false;
    }
    if (tid < 32) {
      // d-1 rotations restore the triangle; lane j updates column j of the
      // two rows a rotation touches
      for (int i = 0; i < d - 1; ++i) {
        const double av = sR[i * SG_SMAX + i], bv = sR[(i + 1) * SG_SMAX + i];
        const double r = hypot(av, bv);
        double c = 1.0, sv = 0.0;
        if (r > 0.0) { c = fabs(av) / r; sv = (av >= 0.0 ? 1.0 : -1.0) * bv / r; }
        __syncwarp();
        const int j = tid;
        if (j >= i && j < d - 1) {
          const double u = sR[i * SG_SMAX + j], w = sR[(i + 1) * SG_SMAX + j];
          sR[i * SG_SMAX + j] = c * u + sv * w;
          sR[(i + 1) * SG_SMAX + j] = -sv * u + c * w;
        }
        if (tid == 0) { s_cr[i] = c; s_sr[i] = sv; }
        __syncwarp();
      }
      // new_i = c L_i + s L_{i+1}, carry = -s L_i + c L_{i+1} on the true
      // columns L = scale * stored; lane i forms the coefficients of rotation i
      const int i = tid;
      if (i < d - 1) {
        const double c = s_cr[i], sv = s_sr[i], sn = s_sc[i + 1];
        // Plain form: the carry holds true values, the incoming stored
        // column N has scale sn.
        gr.q[0][i] = (T)c;
        gr.q[1][i] = (T)(sv * sn);
        gr.q[2][i] = (T)(-sv);
        gr.q[3][i] = (T)(c * sn);
        // Factored form: the stored carry C has scale sc (the chain of the
        // rotations before this one).  Taking out the larger of |c|, |s|
        // keeps every scale factor within [1/sqrt2, 1]:
        //   |c| >= |s|: new = c sc (C + k1 N),  carry = c sn (N + k2 C)
        //   |s| >  |c|: new = s sn (N + k1 C),  carry = -s sc (C + k2 N)
        double sc = s_sc[0];
        for (int k = 0; k < i; ++k)
          sc = fabs(s_cr[k]) >= fabs(s_sr[k]) ? s_cr[k] * s_sc[k + 1] : -s_sr[k] * sc;
        if (fabs(c) >= fabs(sv)) {
          gr.swap[i] = 0;
          gr.k1[i] = (T)(sv * sn / (c * sc));
          gr.k2[i] = (T)(-sv * sc / (c * sn));
          s_scale[i] = fast ? c * sc : 1.0;
        } else {
          gr.swap[i] = 1;
          gr.k1[i] = (T)(c * sc / (sv * sn));
          gr.k2[i] = (T)(-c * sn / (sv * sc));
          s_scale[i] = fast ? sv * sn : 1.0;
        }
      }
      if (tid == 0) gr.sc0 = (T)s_sc[0];
    }
  }
  if (rot) {
    __syncthreads();
    d -= 1;   // columns the new vector is projected on
  }
  double v[RV], tot[RV];
#pragma unroll
  for (int j = 0; j < RV; ++j) v[j] = 0.0;
  if (rot) {
#define SG_CALL(D) givens_body<T, D, EN>(a, gr, fast, v)
    SG_COLS_DISPATCH_UPTO(DMAX - 1, d, SG_CALL)   // d - 1 < M <= DMAX rotations
#undef SG_CALL
  } else {
#define SG_CALL(D) dots_body<T, D>(EN ? a.X : a.B, a.stride, a.t, a.n, v)
    SG_COLS_DISPATCH_UPTO(DMAX, d, SG_CALL)
#undef SG_CALL
  }
  v[DMAX] = (double)vdot<T>(EN ? a.v : a.t, a.t, a.n);
  if (grid_reduce_last<RV>(v, a.partials, &a.st->counter[0], sred, tot)) {
    if (tid == 0) {
      ProjState* st = a.st;
      if (rot) {
        for (int i = 0; i < SG_SMAX * SG_SMAX; ++i) st->R[i] = 0.0;
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j) st->R[i * SG_SMAX + j] = sR[i * SG_SMAX + j];
        for (int j = 0; j < SG_SMAX; ++j) st->scale[j] = (j < d) ? s_scale[j] : 1.0;
        for (int j = 0; j < d; ++j) st->c1[j] = s_scale[j] * tot[j];
      } else {
        for (int j = 0; j < d; ++j) st->c1[j] = st->scale[j] * tot[j];
      }
      st->d = d;
      st->rotated = rot;
      st->nrm0sq = tot[DMAX];
    }
  }
}

// t -= sum_j c_j B_j (D columns), then v[j] = B_j . t (energy: X_j . t)
template <typename T, int D, bool EN, int N>
__device__ __forceinline__ void upd2_body(const ProjArgs<T>& a, const T (&c)[SG_SMAX], double (&v)[N]) {
  using V = typename VecT<T>::V;
  constexpr int W = VecT<T>::W;
  T acc[SG_NZ(D)];
#pragma unroll
  for (int j = 0; j < D; ++j) acc[j] = 0;
  const int nv = a.n / W, stride = gridDim.x * blockDim.x;
  int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (!EN && pipelined<T>(D + 1)) {
    pipe_loop<V, D + 1>(nv,
      [&](int i, V (&buf)[D + 1]) {
        buf[D] = reinterpret_cast<const V*>(a.t)[i];
#pragma unroll
        for (int j = 0; j < D; ++j) buf[j] = colv(a.B, a.stride, j)[i];
      },
      [&](int i, V (&buf)[D + 1]) {
        V tv = buf[D];
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
          for (int w = 0; w < W; ++w) vel(tv, w) = fma(-c[j], vel(buf[j], w), vel(tv, w));
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
          for (int w = 0; w < W; ++w) acc[j] = fma(vel(buf[j], w), vel(tv, w), acc[j]);
        reinterpret_cast<V*>(a.t)[i] = tv;
      });
    i0 = nv;
  }
  for (int i = i0; i < nv; i += stride) {
    V tv = reinterpret_cast<const V*>(a.t)[i];
    V cols[SG_NZ(D)];
#pragma unroll
    for (int j = 0; j < D; ++j) cols[j] = colv(a.B, a.stride, j)[i];
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int w = 0; w < W; ++w) vel(tv, w) -= c[j] * vel(cols[j], w);
    if constexpr (EN) {
#pragma unroll
      for (int j = 0; j < D; ++j) cols[j] = colv(a.X, a.stride, j)[i];
    }
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
      for (int w = 0; w < W; ++w) acc[j] += vel(cols[j], w) * vel(tv, w);
    reinterpret_cast<V*>(a.t)[i] = tv;
  }
  const T* dotcols = EN ? a.X : a.B;
  for (int i = nv * W + blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    T tt = a.t[i];
#pragma unroll
    for (int j = 0; j < D; ++j) tt -= c[j] * a.B[(size_t)j * a.stride + i];
#pragma unroll
    for (int j = 0; j < D; ++j) acc[j] += dotcols[(size_t)j * a.stride + i] * tt;
    a.t[i] = tt;
  }
#pragma unroll
  for (int j = 0; j < D; ++j) v[j] = (double)acc[j];
}

// update sweep 2: t -= B~ c1; c2 = B~^T t (energy: X~^T t)
template <typename T, bool EN, int DMAX>
__global__ void __launch_bounds__(256) k_proj_upd2(const ProjArgs<T> a) {
  __shared__ double sred[32 * DMAX];
  const int d = a.st->d;
  T c[SG_SMAX];
#pragma unroll
  for (int j = 0; j < SG_SMAX; ++j) c[j] = (j < d) ? (T)(a.st->c1[j] * a.st->scale[j]) : (T)0;
  double v[DMAX], tot[DMAX];
#pragma unroll
  for (int j = 0; j < DMAX; ++j) v[j] = 0.0;
#define SG_CALL(D) upd2_body<T, D, EN>(a, c, v)
  SG_COLS_DISPATCH_UPTO(DMAX, d, SG_CALL)
#undef SG_CALL
  if (grid_reduce_last<DMAX>(v, a.partials, &a.st->counter[0], sred, tot)) {
    if (threadIdx.x == 0)
      for (int j = 0; j < d; ++j) a.st->c2[j] = a.st->scale[j] * tot[j];
  }
}

// b~ = t - sum c2_j B_j -> Bd; x~ = x - sum cx_j X_j -> Xd; returns ||b~||^2
// (energy: ||x~||_A^2 = x~ . b~)
template <typename T, int D, bool EN>
__device__ __forceinline__ T upd3_body(const ProjArgs<T>& a, const T (&c2)[SG_SMAX], const T (&cx)[SG_SMAX],
                                       T* Bd, T* Xd) {
  using V = typename VecT<T>::V;
  constexpr int W = VecT<T>::W;
  T nn = 0;
  const int nv = a.n / W, stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    V tv = reinterpret_cast<const V*>(a.t)[i];
    V xv = reinterpret_cast<const V*>(a.v)[i];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const V bc = colv(a.B, a.stride, j)[i];
      const V xc = colv(a.X, a.stride, j)[i];
#pragma unroll
      for (int w = 0; w < W; ++w) {
        vel(tv, w) -= c2[j] * vel(bc, w);
        vel(xv, w) -= cx[j] * vel(xc, w);
      }
    }
#pragma unroll
    for (int w = 0; w < W; ++w) nn += vel(EN ? xv : tv, w) * vel(tv, w);
    reinterpret_cast<V*>(Bd)[i] = tv;
    reinterpret_cast<V*>(Xd)[i] = xv;
  }
  for (int i = nv * W + blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
    T tt = a.t[i], xx = a.v[i];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      tt -= c2[j] * a.B[(size_t)j * a.stride + i];
      xx -= cx[j] * a.X[(size_t)j * a.stride + i];
    }
    nn += (EN ? xx : tt) * tt;
    Bd[i] = tt;
    Xd[i] = xx;
  }
  return nn;
}

// update sweep 3: b~ = t - B~ c2 -> B~ slot d; x~ = x_k - X~ (c1 + c2) -> X~ slot d;
// ||b~||^2 (energy: ||x~||_A^2); acceptance test and R column (Algorithm 2,
// last block)
template <typename T, bool EN, int DMAX>
__global__ void __launch_bounds__(256) k_proj_upd3(const ProjArgs<T> a) {
  __shared__ double sred[32 * NV];
  const int d = a.st->d;
  T c2[SG_SMAX], cx[SG_SMAX];
#pragma unroll
  for (int j = 0; j < SG_SMAX; ++j) {
    c2[j] = (j < d) ? (T)(a.st->c2[j] * a.st->scale[j]) : (T)0;
    cx[j] = (j < d) ? (T)((a.st->c1[j] + a.st->c2[j]) * a.st->scale[j]) : (T)0;
  }
  T* Bd = a.B + (size_t)d * a.stride;
  T* Xd = a.X + (size_t)d * a.stride;
  T nn = 0;
#define SG_CALL(D) nn = upd3_body<T, D, EN>(a, c2, cx, Bd, Xd)
  SG_COLS_DISPATCH_UPTO(DMAX, d, SG_CALL)
#undef SG_CALL
  double v[1] = {(double)nn}, tot[1];
  if (grid_reduce_last<1>(v, a.partials, &a.st->counter[0], sred, tot)) {
    if (threadIdx.x == 0) {
      ProjState* st = a.st;
      // energy: x~ . A x~ can round below zero for a dependent vector
      const double nb = tot[0] > 0.0 ? sqrt(tot[0]) : 0.0;
      st->nrmsq = tot[0];
      const double nrm0 = st->nrm0sq > 0.0 ? sqrt(st->nrm0sq) : 0.0;
      const bool accept = (d == 0) ? (nb > 0.0) : (nb > a.eps_rel * nrm0);
      st->accepted = accept ? 1 : 0;
      if (accept && isfinite(nb)) {
        for (int j = 0; j < d; ++j) st->R[j * SG_SMAX + d] = st->c1[j] + st->c2[j];
        st->R[d * SG_SMAX + d] = nb;
        st->scale[d] = 1.0 / nb;
        st->d = d + 1;
      }
    }
  }
}

__global__ void k_proj_init(ProjState* st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->d = 0; st->accepted = 0; st->rotated = 0;
    for (int i = 0; i < SG_SMAX * SG_SMAX; ++i) st->R[i] = 0.0;
    for (int j = 0; j < SG_SMAX; ++j) { st->scale[j] = 1.0; st->c1[j] = st->c2[j] = st->alpha[j] = 0.0; }
    st->nrm0sq = st->nrmsq = 0.0;
    for (int i = 0; i < 4; ++i) st->counter[i] = 0u;
  }
}

// ---------------------------------------------------------------- host side
namespace {

bool is_ring(int m) { return m == SG_EXTRAP || m == SG_SPEXTRAP || m == SG_LAST; }
bool is_proj(int m) { return m == SG_PROJ_QR || m == SG_PROJ_CLASSIC || m == SG_PROJ_ENERGY; }

int reduce_blocks(int64_t n, int W) {
  int64_t b = ((n + W - 1) / W + 255) / 256;
  int64_t cap = 4LL * sg_num_sms();
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

// Blocks for a grid-stride reduction kernel: at most one wave of resident
// CTAs (the CTAs of a second wave would repeat the per-CTA set-up after the
// first wave has drained), at most the reduce_blocks count the partials
// buffer holds.
template <typename K>
int one_wave(K kernel, int nb, int& cached) {
  if (cached == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    cached = per_sm * sg_num_sms();
  }
  return nb < cached ? nb : cached;
}

struct GuessLayout { size_t state, partials, a, b, t, slot, total; int blocks, nsl; };

GuessLayout guess_layout(int64_t n, int s, int method, int dtype) {
  GuessLayout L{};
  const size_t es = dtype == SG_F64 ? 8 : 4;
  const int W = dtype == SG_F64 ? 2 : 4;
  L.slot = align_up(es * (size_t)n);
  L.blocks = reduce_blocks(n, W);
  L.nsl = (method == SG_LAST) ? 1 : s;
  size_t off = 0;
  L.state = off; off += align_up(sizeof(ProjState));
  L.partials = off; off += align_up(sizeof(double) * NV * (size_t)L.blocks);
  L.a = off;
  if (is_ring(method)) { off += L.slot * L.nsl; L.b = off; L.t = off; }
  else if (is_proj(method)) { off += L.slot * s; L.b = off; off += L.slot * s; L.t = off; off += L.slot; }
  else { L.b = off; L.t = off; }
  L.total = off;
  return L;
}

template <typename T>
ProjArgs<T> proj_args(sg_guess_t g) {
  ProjArgs<T> a{};
  a.B = reinterpret_cast<T*>(g->ws + g->off_a);
  a.X = reinterpret_cast<T*>(g->ws + g->off_b);
  a.t = reinterpret_cast<T*>(g->ws + g->off_t);
  a.stride = g->slot_bytes / sizeof(T);
  a.n = (int)g->n;
  a.M = g->s;
  a.classic = g->method == SG_PROJ_CLASSIC;
  a.energy = g->method == SG_PROJ_ENERGY;
  a.eps_rel = g->eps_rel;
  a.st = reinterpret_cast<ProjState*>(g->ws + g->off_state);
  a.partials = reinterpret_cast<double*>(g->ws + g->off_partials);
  return a;
}

template <typename T>
int extrap_form(sg_guess_t g, void* x0, cudaStream_t s) {
  if (g->count == 0) return SG_OK;
  ExtrapArgs<T> a{};
  const int k = g->count;
  const double* beta = g->beta_tab[k];
  int nt = 0;
  for (int i = 0; i < k; ++i) {   // i = 0 oldest
    if (beta[i] == 0.0) continue;   // sparse extrapolation: skip zero terms
    int slot = ((g->next - k + i) % g->nsl + g->nsl) % g->nsl;
    a.src[nt] = reinterpret_cast<const T*>(g->ws + g->off_a + (size_t)slot * g->slot_bytes);
    a.beta[nt] = beta[i];
    ++nt;
  }
  a.k = nt;
  ProfScope ps(PROF_EXTRAP, s);
  // FP32: up to 8 CTAs of 256 per SM (one wave); FP64 (pipelined): 2 per SM
  int nb = reduce_blocks(g->n, VecT<T>::W) * 2;
  if (pipelined<T>(nt) && nb > PIPE_CTAS_PER_SM * sg_num_sms()) nb = PIPE_CTAS_PER_SM * sg_num_sms();
  T* out = static_cast<T*>(x0);
  const int n = (int)g->n;
#define SG_CALL(K) k_extrap<T, K><<<nb, 256, 0, s>>>(out, a, n)
  switch (nt) {
    case 1: SG_CALL(1); break;   case 2: SG_CALL(2); break;   case 3: SG_CALL(3); break;
    case 4: SG_CALL(4); break;   case 5: SG_CALL(5); break;   case 6: SG_CALL(6); break;
    case 7: SG_CALL(7); break;   case 8: SG_CALL(8); break;   case 9: SG_CALL(9); break;
    case 10: SG_CALL(10); break; case 11: SG_CALL(11); break; case 12: SG_CALL(12); break;
    case 13: SG_CALL(13); break; case 14: SG_CALL(14); break; case 15: SG_CALL(15); break;
    case 16: SG_CALL(16); break; default: return sg_fail(SG_ERR_INVALID, "extrap: bad term count");
  }
#undef SG_CALL
  SG_LAUNCH_CHECK("k_extrap");
  return SG_OK;
}

template <typename T>
int proj_form(sg_guess_t g, const void* b, void* x0, cudaStream_t s) {
  ProjArgs<T> a = proj_args<T>(g);
  a.v = static_cast<const T*>(b);
  a.out = static_cast<T*>(x0);
  const int nb0 = reduce_blocks(g->n, VecT<T>::W);
  // FP64 sweeps are pipelined (two register sets): PIPE_CTAS_PER_SM per SM
  const int nb = sizeof(T) == 8 ? std::min(nb0, PIPE_CTAS_PER_SM * sg_num_sms()) : nb0;
  {
    ProfScope ps(PROF_PROJ_DOTS, s);
    static int w4 = 0, w8 = 0, w16 = 0;
    if (g->s <= 4) k_proj_dots<T, 4><<<one_wave(k_proj_dots<T, 4>, nb, w4), 256, 0, s>>>(a);
    else if (g->s <= 8) k_proj_dots<T, 8><<<one_wave(k_proj_dots<T, 8>, nb, w8), 256, 0, s>>>(a);
    else k_proj_dots<T, 16><<<one_wave(k_proj_dots<T, 16>, nb, w16), 256, 0, s>>>(a);
    SG_LAUNCH_CHECK("k_proj_dots");
  }
  {
    ProfScope ps(PROF_PROJ_LINCOMB, s);
    const int nl = sizeof(T) == 8 ? nb : nb0 * 2;
    if (g->s <= 4) k_proj_lincomb<T, 4><<<nl, 256, 0, s>>>(a);
    else if (g->s <= 8) k_proj_lincomb<T, 8><<<nl, 256, 0, s>>>(a);
    else k_proj_lincomb<T, 16><<<nl, 256, 0, s>>>(a);
    SG_LAUNCH_CHECK("k_proj_lincomb");
  }
  return SG_OK;
}

template <typename T, bool EN, int DMAX>
int proj_update_sweeps(const ProjArgs<T>& a, int nb, cudaStream_t s) {
  static int w1 = 0, w2 = 0, w3 = 0;
  // FP64 rotation and CGS sweeps are pipelined (two register sets): PIPE_CTAS_PER_SM per SM
  const int np = sizeof(T) == 8 ? std::min(nb, PIPE_CTAS_PER_SM * sg_num_sms()) : nb;
  k_proj_upd1<T, EN, DMAX><<<one_wave(k_proj_upd1<T, EN, DMAX>, np, w1), 256, 0, s>>>(a);
  SG_LAUNCH_CHECK("k_proj_upd1");
  k_proj_upd2<T, EN, DMAX><<<one_wave(k_proj_upd2<T, EN, DMAX>, np, w2), 256, 0, s>>>(a);
  SG_LAUNCH_CHECK("k_proj_upd2");
  k_proj_upd3<T, EN, DMAX><<<one_wave(k_proj_upd3<T, EN, DMAX>, nb, w3), 256, 0, s>>>(a);
  SG_LAUNCH_CHECK("k_proj_upd3");
  return SG_OK;
}

template <typename T>
int proj_update(sg_guess_t g, const void* x, cudaStream_t s) {
  ProjArgs<T> a = proj_args<T>(g);
  a.v = static_cast<const T*>(x);
  int rc = sg_sem_apply(g->op, x, a.t, s);
  if (rc) return rc;
  const int nb = reduce_blocks(g->n, VecT<T>::W);
  ProfScope ps(PROF_PROJ_UPDATE, s);
  if (a.energy) {
    if (g->s <= 4) return proj_update_sweeps<T, true, 4>(a, nb, s);
    if (g->s <= 8) return proj_update_sweeps<T, true, 8>(a, nb, s);
    return proj_update_sweeps<T, true, 16>(a, nb, s);
  }
  if (g->s <= 4) return proj_update_sweeps<T, false, 4>(a, nb, s);
  if (g->s <= 8) return proj_update_sweeps<T, false, 8>(a, nb, s);
  return proj_update_sweeps<T, false, 16>(a, nb, s);
}

}  // namespace

extern "C" size_t sg_guess_workspace_bytes(int64_t n, int s, int method, int dtype) {
  if (n < 1 || s < 1 || s > SG_SMAX || method < 0 || method > 6 || (dtype != SG_F64 && dtype != SG_F32)) return 0;
  return guess_layout(n, s, method, dtype).total;
}

extern "C" int sg_guess_create(sg_guess_t* out, int64_t n, int s, int method, int degree_m,
                               double eps_rel, sg_op_t op, void* workspace, int dtype) {
  if (!out) return sg_fail(SG_ERR_INVALID, "guess_create: NULL output handle");
  *out = nullptr;
  if (n < 1 || n >= (1LL << 31)) return sg_fail(SG_ERR_INVALID, "guess_create: n out of range");
  if (s < 1 || s > SG_SMAX) return sg_fail(SG_ERR_INVALID, "guess_create: s must be in [1, 16]");
  if (method < 0 || method > 6) return sg_fail(SG_ERR_INVALID, "guess_create: unknown method");
  if (dtype != SG_F64 && dtype != SG_F32) return sg_fail(SG_ERR_INVALID, "guess_create: bad dtype");
  if (is_proj(method)) {
    if (!op) return sg_fail(SG_ERR_INVALID, "guess_create: projection needs the operator");
    if (op->n != n || op->dtype != dtype) return sg_fail(SG_ERR_INVALID, "guess_create: operator size/dtype mismatch");
    if (!(eps_rel >= 0.0)) return sg_fail(SG_ERR_INVALID, "guess_create: eps_rel must be >= 0");
  }
  int m = degree_m;
  if (m < 0) { m = 0; while ((m + 1) * (m + 1) <= s) ++m; }   // floor(sqrt(s))
  if ((method == SG_EXTRAP || method == SG_SPEXTRAP) && m > s - 1)
    return sg_fail(SG_ERR_INVALID, "guess_create: degree m must be <= s-1");
  GuessLayout L = guess_layout(n, s, method, dtype);
  if (L.total > 0 && !workspace) return sg_fail(SG_ERR_INVALID, "guess_create: NULL workspace");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0)
    return sg_fail(SG_ERR_INVALID, "guess_create: workspace must be 256-byte aligned");
  sg_guess_s* g = new sg_guess_s();
  g->method = method; g->s = s; g->m = m; g->dtype = dtype; g->n = n;
  g->eps_rel = eps_rel; g->op = op;
  g->ws = static_cast<unsigned char*>(workspace);
  g->off_state = L.state; g->off_partials = L.partials; g->off_a = L.a; g->off_b = L.b; g->off_t = L.t;
  g->slot_bytes = L.slot; g->blocks = L.blocks; g->nsl = L.nsl;
  g->count = 0; g->next = 0;
  std::memset(g->beta_tab, 0, sizeof(g->beta_tab));
  if (method == SG_LAST) {
    g->beta_tab[1][0] = 1.0;
  } else if (method == SG_EXTRAP || method == SG_SPEXTRAP) {
    for (int k = 1; k <= s; ++k) {
      int mk = m < k - 1 ? m : k - 1;
      int rc = (method == SG_EXTRAP) ? sgb::lsq_beta(k, mk, g->beta_tab[k])
                                     : sgb::sparse_beta(k, mk, g->beta_tab[k]);
      if (rc) { delete g; return sg_fail(SG_ERR_INVALID, "guess_create: coefficient computation failed"); }
    }
  }
  cudaError_t e = cudaMemsetAsync(g->ws, 0, L.total, 0);
  if (e == cudaSuccess && is_proj(method)) {
    k_proj_init<<<1, 32>>>(reinterpret_cast<ProjState*>(g->ws + g->off_state));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) { delete g; return sg_fail(SG_ERR_CUDA, std::string("guess_create: ") + cudaGetErrorString(e)); }
  *out = g;
  return SG_OK;
}

extern "C" int sg_guess_destroy(sg_guess_t g) { delete g; return SG_OK; }

extern "C" void* sg_guess_next_slot(sg_guess_t g) {
  if (!g || !is_ring(g->method)) return nullptr;
  return g->ws + g->off_a + (size_t)g->next * g->slot_bytes;
}

extern "C" int sg_guess_form(sg_guess_t g, const void* b, void* x0, void* stream) {
  if (!g || !x0) return sg_fail(SG_ERR_INVALID, "guess_form: NULL argument");
  if (!aligned16(x0) || (b && !aligned16(b))) return sg_fail(SG_ERR_INVALID, "guess_form: vectors must be 16-byte aligned");
  cudaStream_t s = as_stream(stream);
  const size_t es = g->dtype == SG_F64 ? 8 : 4;
  if (g->method == SG_ZERO) {
    SG_CUDA_TRY(cudaMemsetAsync(x0, 0, es * (size_t)g->n, s));
    return SG_OK;
  }
  if (is_ring(g->method))
    return g->dtype == SG_F64 ? extrap_form<double>(g, x0, s) : extrap_form<float>(g, x0, s);
  if (!b) return sg_fail(SG_ERR_INVALID, "guess_form: projection needs b");
  return g->dtype == SG_F64 ? proj_form<double>(g, b, x0, s) : proj_form<float>(g, b, x0, s);
}

extern "C" int sg_guess_update(sg_guess_t g, const void* x, const void* b, void* stream) {
  (void)b;
  if (!g || !x) return sg_fail(SG_ERR_INVALID, "guess_update: NULL argument");
  if (!aligned16(x)) return sg_fail(SG_ERR_INVALID, "guess_update: x must be 16-byte aligned");
  cudaStream_t s = as_stream(stream);
  if (g->method == SG_ZERO) return SG_OK;
  if (is_ring(g->method)) {
    void* slot = sg_guess_next_slot(g);
    if (slot != x)
      SG_CUDA_TRY(cudaMemcpyAsync(slot, x, (g->dtype == SG_F64 ? 8 : 4) * (size_t)g->n,
                                  cudaMemcpyDeviceToDevice, s));
    g->next = (g->next + 1) % g->nsl;
    if (g->count < g->nsl) g->count += 1;
    return SG_OK;
  }
  return g->dtype == SG_F64 ? proj_update<double>(g, x, s) : proj_update<float>(g, x, s);
}

// ---------------------------------------------------------------- checkpoint
// Host image of a guess handle: a header (handle parameters and the ring
// position the host keeps) followed by the workspace bytes (history columns,
// projection state and R on the device).
namespace {
struct GuessImageHeader {
  uint64_t magic;
  int64_t n;
  int32_t method, s, m, dtype, count, next;
  uint64_t ws_bytes;
  double eps_rel;                 // projection acceptance threshold
  int32_t op_ex, op_ey, op_ez, op_p, op_dtype, pad;   // projection: the operator of A X~ = B~
  double op_lambda;
};
constexpr uint64_t kGuessImageMagic = 0x5347475545535332ull;

// The image's operator fields: a projection history is orthonormal only under
// the operator (mesh, degree, lambda) it was built with; the EXTRAP family has
// none (zeros).
void image_op_fields(sg_guess_t g, GuessImageHeader& h) {
  h.op_ex = h.op_ey = h.op_ez = h.op_p = h.op_dtype = h.pad = 0;
  h.op_lambda = 0.0;
  if (is_proj(g->method) && g->op) {
    h.op_ex = g->op->g.ex; h.op_ey = g->op->g.ey; h.op_ez = g->op->g.ez; h.op_p = g->op->g.p;
    h.op_dtype = g->op->dtype; h.op_lambda = g->op->lambda;
  }
}
}  // namespace

extern "C" size_t sg_guess_image_bytes(sg_guess_t g) {
  if (!g) return 0;
  return sizeof(GuessImageHeader) + guess_layout(g->n, g->s, g->method, g->dtype).total;
}

extern "C" int sg_guess_export(sg_guess_t g, void* image, void* stream) {
  if (!g || !image) return sg_fail(SG_ERR_INVALID, "guess_export: NULL argument");
  const size_t total = guess_layout(g->n, g->s, g->method, g->dtype).total;
  GuessImageHeader h{};
  h.magic = kGuessImageMagic;
  h.n = g->n; h.method = g->method; h.s = g->s; h.m = g->m; h.dtype = g->dtype;
  h.count = g->count; h.next = g->next; h.ws_bytes = total;
  h.eps_rel = g->eps_rel;
  image_op_fields(g, h);
  std::memcpy(image, &h, sizeof(h));
  cudaStream_t s = as_stream(stream);
  if (total > 0)
    SG_CUDA_TRY(cudaMemcpyAsync(static_cast<unsigned char*>(image) + sizeof(h), g->ws, total,
                                cudaMemcpyDeviceToHost, s));
  SG_CUDA_TRY(cudaStreamSynchronize(s));
  return SG_OK;
}

extern "C" int sg_guess_import(sg_guess_t g, const void* image, size_t image_bytes, void* stream) {
  if (!g || !image) return sg_fail(SG_ERR_INVALID, "guess_import: NULL argument");
  const size_t total = guess_layout(g->n, g->s, g->method, g->dtype).total;
  if (image_bytes != sizeof(GuessImageHeader) + total)
    return sg_fail(SG_ERR_INVALID, "guess_import: image of " + std::to_string(image_bytes) + " bytes, this handle's is " +
                                   std::to_string(sizeof(GuessImageHeader) + total));
  GuessImageHeader h;
  std::memcpy(&h, image, sizeof(h));
  if (h.magic != kGuessImageMagic) return sg_fail(SG_ERR_INVALID, "guess_import: not a guess image");
  if (h.n != g->n || h.method != g->method || h.s != g->s || h.m != g->m || h.dtype != g->dtype ||
      h.ws_bytes != total)
    return sg_fail(SG_ERR_INVALID, "guess_import: image of a handle with other n, s, method, degree or dtype");
  // ring position: update keeps count = min(k, nsl) and next = k mod nsl after
  // k updates, so next == count until the ring is full; projection handles keep
  // both at 0 (their state is on the device)
  const bool ring = is_ring(g->method);
  const bool pos_ok = ring ? (h.count >= 0 && h.count <= g->nsl && h.next >= 0 && h.next < g->nsl &&
                              (h.count == g->nsl || h.next == h.count))
                           : (h.count == 0 && h.next == 0);
  if (!pos_ok) return sg_fail(SG_ERR_INVALID, "guess_import: ring position out of range (corrupt image)");
  GuessImageHeader mine{};
  image_op_fields(g, mine);
  if (is_proj(g->method) &&
      (h.eps_rel != g->eps_rel || h.op_ex != mine.op_ex || h.op_ey != mine.op_ey || h.op_ez != mine.op_ez ||
       h.op_p != mine.op_p || h.op_dtype != mine.op_dtype || h.op_lambda != mine.op_lambda))
    return sg_fail(SG_ERR_INVALID, "guess_import: projection image built with another operator or eps_rel");
  cudaStream_t s = as_stream(stream);
  if (total > 0)
    SG_CUDA_TRY(cudaMemcpyAsync(g->ws, static_cast<const unsigned char*>(image) + sizeof(h), total,
                                cudaMemcpyHostToDevice, s));
  SG_CUDA_TRY(cudaStreamSynchronize(s));
  g->count = h.count;
  g->next = h.next;
  return SG_OK;
}

extern "C" int sg_guess_info(sg_guess_t g, int* d, double* R, void* stream) {
  if (!g) return sg_fail(SG_ERR_INVALID, "guess_info: NULL handle");
  cudaStream_t s = as_stream(stream);
  if (is_proj(g->method)) {
    ProjState h;
    SG_CUDA_TRY(cudaMemcpyAsync(&h, g->ws + g->off_state, sizeof(ProjState), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaStreamSynchronize(s));
    if (d) *d = h.d;
    if (R)
      for (int i = 0; i < g->s; ++i)
        for (int j = 0; j < g->s; ++j) R[i * g->s + j] = h.R[i * SG_SMAX + j];
    return SG_OK;
  }
  if (d) *d = g->count;
  if (R) {
    for (int i = 0; i < g->s; ++i) R[i] = 0.0;
    for (int i = 0; i < g->count && i < g->s; ++i) R[i] = g->beta_tab[g->count][i];
  }
  return SG_OK;
}
