// sg_common.cuh -- internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/sg.h"

#define SG_PMAX SG_MAX_DEGREE   // largest GLL degree
#define SG_SMAX SG_MAX_HISTORY  // largest history size

// ---------------------------------------------------------------- errors
void sg_set_error(const std::string& msg);
int sg_fail(int code, const std::string& msg);

#define SG_CUDA_TRY(call)                                                        \
  do {                                                                          \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess)                                                       \
      return sg_fail(SG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void sg_count_launch();
void sg_count_launches(long long n);   // kernels a graph launch ran

#define SG_LAUNCH_CHECK(name)                                                    \
  do {                                                                          \
    sg_count_launch();                                                           \
    cudaError_t e_ = cudaGetLastError();                                         \
    if (e_ != cudaSuccess)                                                       \
      return sg_fail(SG_ERR_CUDA, std::string("launch ") + name + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------- profiling
enum { PROF_SEM = 0, PROF_PCG_APPLY = 1, PROF_PCG_UPDATE = 2, PROF_EXTRAP = 3,
       PROF_PROJ_DOTS = 4, PROF_PROJ_LINCOMB = 5, PROF_PROJ_UPDATE = 6, PROF_N = 7 };
struct ProfScope {   // records an event pair around one launch when profiling is on
  int id; cudaStream_t s; int active;
  ProfScope(int id_, cudaStream_t s_);
  ~ProfScope();
};

// ---------------------------------------------------------------- fast divmod
// Division by a run-time invariant d (Granlund & Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994): for n < 2^31,
// q = (umulhi(n, m) + n) >> s with s = ceil(log2 d), m = 2^32 (2^s - d) / d + 1.
struct FastDiv {
  uint32_t d, m, s;
  __host__ __device__ FastDiv() : d(1), m(1), s(0) {}
  __host__ FastDiv(uint32_t d_) : d(d_) {
    s = 0;
    while ((1ull << s) < d) ++s;
    m = (uint32_t)(((1ull << 32) * ((1ull << s) - d)) / d + 1);
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    return (__umulhi(n, m) + n) >> s;
  }
  __host__ uint32_t div_host(uint32_t n) const {
    return (uint32_t)((((uint64_t)n * m) >> 32) + n) >> s;
  }
};

// ---------------------------------------------------------------- operator
// Geometry and 1D coefficient tables of the assembled affine-box operator.
//
// On a box mesh of equal axis-aligned elements the element operator of
// Sec. 5.1 is a sum of Kronecker products, a_x Khat (x) W (x) W + ..., and
// the gather-scatter of a Kronecker product over a tensor-product numbering
// is the Kronecker product of the assembled 1D matrices.  So A = sum_dir
// a_dir K1 (x) W1 (x) W1 + c_m W1 (x) W1 (x) W1 exactly, with K1 the
// assembled 1D GLL stiffness (bandwidth p) and W1 the assembled 1D mass.
// Written with the weights factored out of each row:
//   (A u)_ijk = W_i W_j W_k [ sum_dir (C_dir u)_along-dir + c_m u_ijk ],
// C_dir = a_dir diag(W1)^-1 K1 -- rows by local index a = i mod p:
//   C[a][l]  (a = 1..p-1) : a_dir Khat[a][l] / w_a, on element e's line
//   C[0][l]               : a_dir Khat[0][l] / (w_0 + w_p), element e
//   C[p][l]               : a_dir Khat[p][l] / (w_0 + w_p), element e-1
struct SemGeom {
  int nx, ny, nz;          // global nodes per axis (p*e + 1)
  int ex, ey, ez, p;
  double cm;               // lambda * hx hy hz / 8
  double adir[3];          // direction factors J (2/h_d)^2 = (hx hy hz / h_d^2) / 2
  double C[3][SG_PMAX + 1][SG_PMAX + 1];  // per direction x, y, z
  double wl[SG_PMAX + 1];  // assembled 1D mass by local index (wl[0] = w0 + wp)
  double dg[3][SG_PMAX + 1];              // diagonal coefficient by local index
  const void* tabs;        // device: the operator kernel's coefficients, SemTabs (sg_op.cu)
  const void* htabs;       // host: the same bytes, passed by value to the operator kernel
  int zl;                  // element layers per operator CTA; 0 = automatic
};

struct sg_op_s {
  int dtype;
  double lambda;
  int64_t n;
  SemGeom g;
  double nodes[SG_PMAX + 1], weights[SG_PMAX + 1];
  FastDiv div_nx, div_nxy;
  int device;
  unsigned long long uid;   // unique per created operator (never reused)
  int last_iters;           // iterations of the last PCG solve (sizes the first chunk)
  void* pcg_graphs;         // cached PCG iteration graphs (sg_pcg.cu), released with the operator
  void* d_tabs;             // device copy of the operator kernel's tables (g.tabs)
  alignas(16) unsigned char htabs[2048];   // host copy (g.htabs), sizeof(SemTabs<T, p>) bytes
};

// Release the PCG iteration graphs cached on an operator (sg_pcg.cu).
void sg_pcg_release(sg_op_s* op);
// True while library-side kernel timing is enabled (sg_profile_enable).
bool sg_profiling_on();

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int ceil_pow2(int v) { int p = 1; while (p < v) p <<= 1; return p; }
constexpr int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }

// Deterministic block sum of NV <= 32 values per thread.  Result valid in
// thread 0.  Warp stage, for NV >= 2 "transposed": the NV values (padded to
// NP, a power of two) are halved every exchange -- a lane keeps the upper or
// the lower half by its lane bit and adds the partner's copy of that half --
// so after log2(NP) exchanges each lane carries the partial sum of one value
// and the remaining 5 - log2(NP) exchanges complete it: NP - 1 + 5 - log2(NP)
// additions per warp instead of 5 NV.  Then warp 0 adds the warp totals in
// warp order.  A block's last warp, when only partly populated, sums each
// value with its own shuffle tree instead (its missing lanes hold no results).
// Summation order is fixed, so results repeat bit for bit.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /* >= 32*NV */) {
  static_assert(NV >= 1 && NV <= 32, "block_sum: 1..32 values");
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int nwarps = (nthreads + 31) >> 5;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int tl = tid & 31, tw = tid >> 5;
  constexpr int NP = ceil_pow2(NV), L = ilog2(NP), G = 32 >> L;   // lanes per value at the end
  const bool full = nthreads - tw * 32 >= 32;
  double t = 0.0;
  const int j = (tl >> (5 - L)) & (NP - 1);   // value a full warp's lane ends with
  if (full) {                        // transposed reduction
    double w[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) w[k] = (k < NV) ? v[k] : 0.0;
#pragma unroll
    for (int r = 0; r < L; ++r) {
      const int o = 16 >> r, half = NP >> (r + 1);
      const bool hi = (tl & o) != 0;
#pragma unroll
      for (int i = 0; i < half; ++i) {
        const double keep = hi ? w[half + i] : w[i];
        const double give = hi ? w[i] : w[half + i];
        w[i] = keep + __shfl_xor_sync(0xffffffffu, give, o);
      }
    }
    t = w[0];
#pragma unroll
    for (int o = G >> 1; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  } else {                           // the block's last, partial warp: one tree per value into lane 0
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  }
  __syncthreads();                   // smem free from any earlier use
  if (full) {
    if ((tl & (G - 1)) == 0 && j < NV) smem[j * 32 + tw] = t;
  } else if (tl == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[k * 32 + tw] = v[k];
  }
  __syncthreads();
  if (tw == 0) {
    double a = 0.0;
    if (tl < NV)
      for (int q = 0; q < nwarps; ++q) a += smem[tl * 32 + q];
    __syncwarp();
    if (tl < NV) smem[tl] = a;
    __syncwarp();
    if (tl == 0) {
#pragma unroll
      for (int k = 0; k < NV; ++k) v[k] = smem[k];
    }
  }
  __syncthreads();
}



// Grid-level deterministic reduction: every block writes its NV partial sums
// to partials[block*NV + k]; the last block to finish sums them in block
// order and returns true (in all of its threads) with the totals in out[]
// (valid in thread 0).  counter must start at 0; it is reset by the last block.
template <int NV>
__device__ bool grid_reduce_last(double (&v)[NV], double* partials, unsigned int* counter,
                                 double* smem, double (&out)[NV]) {
  __shared__ bool s_last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int nblocks = gridDim.x * gridDim.y * gridDim.z;
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  block_sum<NV>(v, smem);
  if (tid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(size_t)bid * NV + k] = v[k];
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == (unsigned int)nblocks - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int b = tid; b < nblocks; b += nthreads) {
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(&partials[(size_t)b * NV + k]);
  }
  block_sum<NV>(acc, smem);
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = acc[k];
  if (tid == 0) *counter = 0u;
  return true;
}

// ---------------------------------------------------------------- launch helpers
int sg_num_sms();
// Relative tolerance of one FP32 inner solve of iterative refinement given
// the outer target tol and the current relative FP64 residual rel.
double ir_inner_tol(double inner_tol, double tol, double rel);
inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
