// sg_sem_kernel.cuh -- the tiled matrix-free SEM operator kernel (Sec. 5.1).
//
// Node-centric form of the assembled affine-box operator (see SemGeom):
//   (A u)_ijk = W_i W_j W_k [ (C_x u)_i + (C_y u)_j + (C_z u)_k + c_m u_ijk ].
// Row a of C_dir (a = local index of the node in its element) touches only
// the nodes of the node's element along that direction, plus, for a = 0 (a
// node shared by elements e-1 and e), those of element e-1.  Each output node
// is therefore computed exactly once, without atomics or a scatter pass.
//
// Tiling: a CTA owns an element-aligned tile of TX x TY nodes in x,y (one
// thread per (x,y) column) and marches through ZL element layers in z.  For
// each layer the p+1 planes z = e p .. e p + p are held in shared memory,
// padded by p nodes below and 1 node above in x and y; the top plane of a
// layer is reused as the bottom plane of the next.  The z-contraction runs in
// registers on the thread's own column; the x- and y-contractions read the
// padded planes.  Nodes with local index p-1... 0 are owned; the upper
// boundary faces (index n-1) are Dirichlet and are written as 0 separately.
//
// MODE 0: out = A x.
// MODE 1: PCG step (Sec. 5.3): p_new = z + beta p_old (p_new = z on the first
//         iteration), out2 = p_new, out = q = A p_new, partial p_new . q;
//         the last CTA forms alpha = (r.z) / (p.q).
// MODE 2: residual: out = r = b - A x, out2 = z = r / diag(A), partials
//         r.r, r.z, b.b; the last CTA stores them (PCG start / true residual).
#pragma once
#include "sg_common.cuh"

struct PcgState {
  double rz, pq, rr, bb, rr0, thr2;
  double alpha, beta;
  double rr_true;
  int iter, done, status, first;
  int maxit, criterion;
  double tol;
  unsigned int counter[4];
  int diag_tag;            // nonzero once inverse diagonal is in the workspace
  int pad[7];
};

enum { PCG_RUNNING = 0, PCG_CONVERGED = 1, PCG_MAXIT = 2, PCG_BREAKDOWN = 3 };

template <int P>
struct SemTile {
  static constexpr int TEX = ((28 + P / 2) / P) > 0 ? ((28 + P / 2) / P) : 1;
  static constexpr int TEY = ((14 + P / 2) / P) > 0 ? ((14 + P / 2) / P) : 1;
  static constexpr int TX = TEX * P, TY = TEY * P;
  static constexpr int PX = TX + P + 1, PY = TY + P + 1, NPL = P + 1;
  static constexpr int CS = P + 2;  // padded row stride of the coefficient tables
  static constexpr int NTHREADS = TX * TY;
};

template <typename T>
struct SemArgs {
  const T* x;     // MODE 0/2: input x     MODE 1: z
  const T* aux;   // MODE 1: p_old          MODE 2: b
  const T* invd;  // MODE 2: 1/diag(A)
  T* out;         // MODE 0: y   MODE 1: q      MODE 2: r
  T* out2;        // MODE 1: p_new            MODE 2: z
  double* partials;
  PcgState* st;
  int zl;         // element layers per CTA
  int final_pass; // MODE 2: 1 = true-residual check (store rr_true only)
};

template <typename T, int P>
__device__ __forceinline__ bool interior_node(const SemGeom& g, int gx, int gy, int gz) {
  return gx > 0 && gy > 0 && gz > 0 && gx < g.nx - 1 && gy < g.ny - 1 && gz < g.nz - 1;
}

template <typename T, int P, int MODE>
__global__ void __launch_bounds__(SemTile<P>::NTHREADS)
k_sem(const SemGeom g, const SemArgs<T> a) {
  using TL = SemTile<P>;
  constexpr int TX = TL::TX, TY = TL::TY, PX = TL::PX, PY = TL::PY, NPL = TL::NPL, CS = TL::CS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);                     // NPL planes of PY x PX
  __shared__ T sC[3][P + 1][CS];
  __shared__ T sW[P + 1];
  __shared__ double sred[32 * 3];
  __shared__ int s_skip;
  __shared__ T s_beta;
  __shared__ int s_first;

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + TX * ty;
  if (MODE == 1) {
    if (tid == 0) {
      s_skip = a.st->done;
      s_beta = (T)a.st->beta;
      s_first = a.st->first;
    }
  }
  for (int i = tid; i < 3 * (P + 1) * (P + 1); i += TL::NTHREADS) {
    int d = i / ((P + 1) * (P + 1)), r = (i / (P + 1)) % (P + 1), c = i % (P + 1);
    sC[d][r][c] = (T)g.C[d][r][c];
  }
  for (int i = tid; i <= P; i += TL::NTHREADS) sW[i] = (T)g.wl[i];
  __syncthreads();
  if (MODE == 1 && s_skip) return;

  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int e0 = blockIdx.z * a.zl;
  const int e1 = min(g.ez, e0 + a.zl);
  const int gx = x0 + tx, gy = y0 + ty;
  const int ia = tx % P, ib = ty % P;
  const bool col_in = (gx < g.nx - 1) && (gy < g.ny - 1);
  const bool col_int = col_in && gx > 0 && gy > 0;
  const T wxy = sW[ia] * sW[ib];
  const T cm = (T)g.cm;
  const size_t nxy = (size_t)g.nx * g.ny;

  // value of the operand at a global point (0 outside the interior)
  auto operand = [&](int px, int py, int pz) -> T {
    if (px <= 0 || py <= 0 || pz <= 0 || px >= g.nx - 1 || py >= g.ny - 1 || pz >= g.nz - 1)
      return (T)0;
    size_t idx = (size_t)px + (size_t)g.nx * py + nxy * pz;
    if (MODE == 1) {
      T zv = a.x[idx];
      return s_first ? zv : zv + s_beta * a.aux[idx];
    }
    return a.x[idx];
  };

  // z-carry from the element below the chunk: its line's contribution to plane e0*P
  T carry = (T)0;
  if (e0 > 0 && col_int) {
    T ub[P + 1];
#pragma unroll
    for (int l = 0; l <= P; ++l) ub[l] = operand(gx, gy, (e0 - 1) * P + l);
#pragma unroll
    for (int l = 0; l <= P; ++l) carry += sC[2][P][l] * ub[l];
  }

  double acc_red[3] = {0.0, 0.0, 0.0};

  for (int e = e0; e < e1; ++e) {
    // ---- stage planes e*P .. e*P + P (the first plane is kept from the last layer)
    __syncthreads();
    const int pl0 = (e == e0) ? 0 : 1;
    for (int pl = pl0; pl <= P; ++pl) {
      const int gz = e * P + pl;
      T* plane = S + (size_t)(gz % NPL) * PY * PX;
      for (int i = tid; i < PY * PX; i += TL::NTHREADS) {
        int py = i / PX, px = i - py * PX;
        plane[i] = operand(x0 - P + px, y0 - P + py, gz);
      }
    }
    __syncthreads();

    T u[P + 1];
#pragma unroll
    for (int l = 0; l <= P; ++l)
      u[l] = S[(size_t)((e * P + l) % NPL) * PY * PX + (ty + P) * PX + (tx + P)];

#pragma unroll
    for (int c = 0; c < P; ++c) {
      const int gz = e * P + c;
      const T* plane = S + (size_t)(gz % NPL) * PY * PX;
      // z-direction: own column, element e (+ carry from element e-1 at c = 0)
      T acc = cm * u[c];
#pragma unroll
      for (int l = 0; l <= P; ++l) acc += sC[2][c][l] * u[l];
      if (c == 0) acc += carry;
      // x-direction
      {
        const T* row = plane + (ty + P) * PX + (tx - ia + P);
#pragma unroll
        for (int l = 0; l <= P; ++l) acc += sC[0][ia][l] * row[l];
        if (ia == 0) {
#pragma unroll
          for (int l = 0; l <= P; ++l) acc += sC[0][P][l] * row[l - P];
        }
      }
      // y-direction
      {
        const T* colp = plane + (ty - ib + P) * PX + (tx + P);
#pragma unroll
        for (int l = 0; l <= P; ++l) acc += sC[1][ib][l] * colp[l * PX];
        if (ib == 0) {
#pragma unroll
          for (int l = 0; l <= P; ++l) acc += sC[1][P][l] * colp[(l - P) * PX];
        }
      }
      const bool inside = col_int && gz > 0;
      T yv = inside ? (wxy * sW[c]) * acc : (T)0;
      if (col_in) {
        size_t idx = (size_t)gx + (size_t)g.nx * gy + nxy * gz;
        if (MODE == 0) {
          a.out[idx] = yv;
        } else if (MODE == 1) {
          T pv = u[c];
          a.out[idx] = yv;
          a.out2[idx] = pv;
          acc_red[0] += (double)pv * (double)yv;
        } else {
          T bv = inside ? a.aux[idx] : (T)0;
          T rv = inside ? bv - yv : (T)0;
          T zv = rv * a.invd[idx];
          a.out[idx] = rv;
          if (!a.final_pass) a.out2[idx] = zv;
          acc_red[0] += (double)rv * (double)rv;
          acc_red[1] += (double)rv * (double)zv;
          acc_red[2] += (double)bv * (double)bv;
        }
      }
    }
    // carry for the next layer: element e's line contribution to plane (e+1)P
    carry = (T)0;
#pragma unroll
    for (int l = 0; l <= P; ++l) carry += sC[2][P][l] * u[l];
  }

  // ---- upper Dirichlet faces (index n-1) inside this CTA's region: write 0
  {
    const bool lastx = (x0 + TX >= g.nx - 1), lasty = (y0 + TY >= g.ny - 1);
    const bool lastz = (e1 == g.ez);
    const int xe = lastx ? g.nx : x0 + TX, ye = lasty ? g.ny : y0 + TY;
    const int z0 = e0 * P, ze = lastz ? g.nz : e1 * P;
    const int wx = xe - x0, wy = ye - y0, wz = ze - z0;
    const int total = wx * wy * wz;
    if (lastx || lasty || lastz) {
      for (int i = tid; i < total; i += TL::NTHREADS) {
        int lx = i % wx, ly = (i / wx) % wy, lz = i / (wx * wy);
        int px = x0 + lx, py = y0 + ly, pz = z0 + lz;
        if (px == g.nx - 1 || py == g.ny - 1 || pz == g.nz - 1) {
          size_t idx = (size_t)px + (size_t)g.nx * py + nxy * pz;
          a.out[idx] = (T)0;
          if (MODE == 1 || (MODE == 2 && !a.final_pass)) a.out2[idx] = (T)0;
        }
      }
    }
  }

  if (MODE == 1) {
    double v[1] = {acc_red[0]}, tot[1];
    if (grid_reduce_last<1>(v, a.partials, &a.st->counter[0], sred, tot)) {
      if (tid == 0) {
        PcgState* st = a.st;
        double pq = tot[0];
        st->pq = pq;
        st->first = 0;
        if (!(pq > 0.0) || !isfinite(pq)) {
          st->status = PCG_BREAKDOWN;
          st->done = 1;
        } else {
          st->alpha = st->rz / pq;
        }
      }
    }
  } else if (MODE == 2) {
    double v[3] = {acc_red[0], acc_red[1], acc_red[2]}, tot[3];
    if (grid_reduce_last<3>(v, a.partials, &a.st->counter[0], sred, tot)) {
      if (tid == 0) {
        PcgState* st = a.st;
        if (a.final_pass) {
          st->rr_true = tot[0];
        } else {
          st->rr = tot[0];
          st->rz = tot[1];
          st->bb = tot[2];
          st->rr0 = tot[0];
          const double tol = st->tol;
          double thr;
          int strict = 1;
          if (st->criterion == SG_STOP_INITRESID) thr = tol * fmax(sqrt(tot[0]), 1.0);
          else if (st->criterion == SG_STOP_RHS) thr = tol * fmax(sqrt(tot[2]), 1.0);
          else { thr = tol * sqrt(tot[2]); strict = 0; }
          st->thr2 = thr * thr;
          st->iter = 0;
          st->first = 1;
          st->beta = 0.0;
          bool conv = strict ? (tot[0] < st->thr2) : (tot[0] <= st->thr2);
          if (!isfinite(tot[0])) { st->status = PCG_BREAKDOWN; st->done = 1; }
          else if (conv) { st->status = PCG_CONVERGED; st->done = 1; }
          else if (st->maxit <= 0) { st->status = PCG_MAXIT; st->done = 1; }
          else { st->status = PCG_RUNNING; st->done = 0; }
        }
      }
    }
  }
}
