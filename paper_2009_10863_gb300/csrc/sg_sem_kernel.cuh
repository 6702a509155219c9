// sg_sem_kernel.cuh -- the tiled matrix-free SEM operator kernel (Sec. 5.1).
//
// Form of the operator (see SemGeom): on the affine box the assembled operator
// is a Kronecker sum of assembled 1D operators,
//   (A u)_ijk = W_i W_j W_k [ (C_x u)_i + (C_y u)_j + (C_z u)_k + c_m u_ijk ],
// where row a of C (a = local index of the node in its element) combines the
// p+1 nodes of the node's element along that direction, and a shared node
// (a = 0) also row p of C on the element before it.
//
// Element-line contractions.  Per direction the kernel applies the (p+1)x(p+1)
// matrix C to each element line (the sum-factorised tensor contraction of the
// paper's local operator).  C is centrosymmetric (C[p-a][p-l] = C[a][l]), so
// each line uses the even-odd split: s_l = u_l + u_{p-l}, d_l = u_l - u_{p-l},
// o_a = E_a + O_a, o_{p-a} = E_a - O_a with two half-size products -- about
// 3/4 of the multiply-adds of the plain product, and no divergent branches
// (the odd sum is accumulated onto E_a, and o_{p-a} = 2 E_a - o_a).
// The contribution of the element before a shared node (row p of C on its
// line) is added by the line that owns the node, so every output node is
// written exactly once, without atomics or a scatter pass.  The weight W_k of
// an output's z index sits in the coefficient tables (sem_tables), so the
// epilogue multiplies by W_i W_j only.
//
// Tiling.  A CTA owns TEX x TEY elements in x,y (TX x TY nodes, one thread per
// (x,y) column) and marches through ZL element layers in z.  For each layer the
// p+1 planes z = e p .. e p + p sit in shared memory, padded by p nodes below
// and 1 above in x and y (the top plane is reused as the next layer's bottom).
// Planes are staged with cp.async (zero-filled outside the interior) into a
// ring of 2p+1 slots, so the next layer's planes load while this one computes;
// a CTA of one layer (FP64) uses the p slots no later layer needs for its
// epilogue operands (old q, p; or b, 1/diag), also by cp.async.
//   z: each thread contracts its own column in registers; the top output of a
//      layer is carried to the next layer's bottom node;
//   x: item (plane c, row y, element) -> p outputs written to a work buffer;
//   y: item (plane c, column x, element) -> p outputs; FP64 adds them to the
//      x results in the same buffer (three barriers per layer), FP32 writes a
//      second buffer (two barriers);
// the thread then adds its column's x and y results (the mass term is in the
// z table), multiplies by W_i W_j, and stores.  The upper Dirichlet faces
// (index n-1) are written 0.
//
// MODE 0: out = A x.
// MODE 1: PCG step (Sec. 5.3) on the staged z: w = A z, then for owned nodes
//         p = z + beta p, q = w + beta q in place (p = z, q = w first), which is
//         q = A p by linearity; p . q -> alpha = (r.z)/(p.q).
// MODE 2: residual: out = r = b - A x, out2 = z = r / diag(A); r.r, r.z, b.b
//         (final_pass: r, r.r and b.b only -- the true residual).
#pragma once
#include <type_traits>

#include "sg_common.cuh"

#ifndef SG_SEM_F32_MINB
#define SG_SEM_F32_MINB 4   // FP32 operator CTAs per SM the register budget is sized for
#endif
#ifndef SG_SEM_F32_PXPAD
#define SG_SEM_F32_PXPAD 0  // extra words per staged row (FP32 shared-memory pitch)
#endif

struct PcgState {
  double rz, pq, rr, bb, rr0, thr2;
  double alpha, beta;
  double rr_true;
  int iter, done, status, first;
  int maxit, criterion;
  double tol;
  unsigned int counter[4];
  unsigned long long diag_tag;   // operator tag of the 1/diag(A) held in the workspace
  void* xvec;                    // solution vector of the running solve (set by the set-up kernel)
  int pad[6];
};

enum { PCG_RUNNING = 0, PCG_CONVERGED = 1, PCG_MAXIT = 2, PCG_BREAKDOWN = 3 };

// Device vectors of one PCG solve's iterations (x == nullptr: the solution
// vector recorded in the state by the solve's set-up).
template <typename T>
struct PcgIterPtrs {
  PcgState* st;
  double* partials;
  T *r, *z, *p, *q, *x;
  const T* invd;
};

template <int P>
struct SemTile {
  static constexpr int TEX = (P <= 2) ? 8 : (P <= 4 ? 4 : 2);
  static constexpr int TEY = (P <= 2) ? 4 : 2;
  static constexpr int TX = TEX * P, TY = TEY * P;
  static constexpr int PX = TX + P + 1, PY = TY + P + 1, NPL = 2 * P + 1;  // ring slots
  static constexpr int NTHREADS = TX * TY;
  // row pitch of a staged plane in shared memory (>= PX; padding moves the
  // rows of the y line items onto other banks)
  template <typename T> static constexpr int pitch() { return sizeof(T) == 4 ? PX + SG_SEM_F32_PXPAD : PX; }
  static constexpr int MINB = (NTHREADS <= 256) ? 3 : 1;   // CTAs per SM to fit registers for
  template <typename T> static constexpr int minb() { return sizeof(T) == 4 ? SG_SEM_F32_MINB : MINB; }
  // separate x and y result buffers (2 barriers per layer instead of 4): FP32 only,
  // where shared memory is not the occupancy limit
  template <typename T> static constexpr bool two_w() { return sizeof(T) == 4; }
  static constexpr int N = P + 1, H = (P + 1) / 2;
  static constexpr bool MID = ((P + 1) % 2) == 1;
  static constexpr int HE = H + (MID ? 1 : 0);   // even-part outputs (incl. middle)
};

template <typename T>
struct SemArgs {
  const T* x;     // staged operand: MODE 0/2: x     MODE 1: z
  const T* aux;   // MODE 2: b
  const T* invd;  // MODE 2: 1/diag(A)
  T* out;         // MODE 0: y   MODE 1: q (in/out)   MODE 2: r
  T* out2;        // MODE 1: p (in/out)             MODE 2: z
  double* partials;
  PcgState* st;
  int zl;         // element layers per CTA (at most; the grid's z chunks are balanced)
  int final_pass; // MODE 2: 1 = true-residual check (store rr_true only)
};

// Even-odd coefficient tables of one direction's C, rows multiplied by the
// assembled mass weights of the output nodes (see sem_tables).
template <typename T, int P>
struct __align__(16) EOTab {
  using TL = SemTile<P>;
  T ce[TL::HE][TL::H];            // (C[a][l] + C[a][p-l]) / 2, a < H (+ middle row)
  T co[TL::H][TL::H];             // (C[a][l] - C[a][p-l]) / 2, a < H
  T crow[P + 1];                  // row p of C: contribution to the next element's node 0
  T cm[TL::MID ? TL::HE : 1];     // C[a][mid] (odd line length only)
};

// Copy n consecutive table entries into registers, 16 bytes per shared-memory
// load when the run is 16-byte aligned and sized (rows of 4 floats or doubles).
template <typename T, int N>
__device__ __forceinline__ void load_run(const T* src, T (&dst)[N]) {
  if constexpr ((N * sizeof(T)) % 16 == 0) {
    constexpr int PER = 16 / sizeof(T);
#pragma unroll
    for (int k = 0; k < N / PER; ++k) {
      const float4 v = reinterpret_cast<const float4*>(src)[k];
      const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
      for (int w = 0; w < PER; ++w) dst[k * PER + w] = e[w];
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) dst[k] = src[k];
  }
}

// The operator's coefficients, built once per operator on the host (sg_op.cu):
//   t[0]  z: C_z + c_m I, row a multiplied by W_a (W_p = W_0) -- the z line
//         products carry the weight W_k of their output nodes;
//   t[1]  x: C_x;   t[2]  y: C_y;
//   w     the assembled 1D mass weights by local index (w[0] = w_0 + w_p).
// The single-system kernel takes them as a kernel parameter: every CTA and
// warp reads the same entries at compile-time offsets, so the line products
// take them as constant-bank operands (no shared-memory table, no loads).  The
// batched kernel keeps a shared-memory copy (its systems differ per item).
template <typename T, int P>
struct __align__(16) SemTabs {
  EOTab<T, P> t[3];
  T w[P + 1];
};

// o[0..P] = C u for one element line (even-odd), coefficients from table t.
// With ROW, o[0] also receives row p of C applied to the line ul of the
// element before (the other element of the shared node 0).
// Per output pair the odd sum starts from the even one, op = E_a + O_a, and
// o[p-a] = 2 E_a - op: one multiply-add instead of a multiply and two adds.
template <typename T, int N, bool SMEM>
__device__ __forceinline__ void table_run(const T* src, T (&dst)[N]) {
  if constexpr (SMEM) {
    load_run<T, N>(src, dst);     // shared memory: 16-byte loads
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) dst[k] = src[k];   // kernel parameter: constant operands
  }
}

template <typename T, int P, bool ROW, bool SMEM>
__device__ __forceinline__ void line_eo(const T (&u)[P + 1], const T (&ul)[P + 1], const EOTab<T, P>& t,
                                        T (&o)[P + 1]) {
  using TL = SemTile<P>;
  constexpr int H = TL::H;
  T s[H], d[H];
#pragma unroll
  for (int l = 0; l < H; ++l) { s[l] = u[l] + u[P - l]; d[l] = u[l] - u[P - l]; }
#pragma unroll
  for (int a = 0; a < H; ++a) {
    T ce[H], co[H];
    table_run<T, H, SMEM>(t.ce[a], ce);
    table_run<T, H, SMEM>(t.co[a], co);
    T e = ce[0] * s[0];
#pragma unroll
    for (int l = 1; l < H; ++l) e = fma(ce[l], s[l], e);
    if constexpr (TL::MID) e = fma(t.cm[a], u[P / 2], e);
    T op = e;
#pragma unroll
    for (int l = 0; l < H; ++l) op = fma(co[l], d[l], op);
    o[P - a] = fma((T)2, e, -op);
    if (ROW && a == 0) {
      T cr[P + 1];
      table_run<T, P + 1, SMEM>(t.crow, cr);
#pragma unroll
      for (int l = 0; l <= P; ++l) op = fma(cr[l], ul[l], op);
    }
    o[a] = op;
  }
  if constexpr (TL::MID) {
    T e = t.cm[H] * u[P / 2];
#pragma unroll
    for (int l = 0; l < H; ++l) e = fma(t.ce[H][l], s[l], e);
    o[P / 2] = e;
  }
}

template <typename T, int P>
__device__ __forceinline__ T row_dot(const T (&u)[P + 1], const EOTab<T, P>& t) {
  T r = t.crow[0] * u[0];
#pragma unroll
  for (int l = 1; l <= P; ++l) r += t.crow[l] * u[l];
  return r;
}

// Table of direction d with row a of C multiplied by rowmul[a] (rowmul[p] =
// rowmul[0] keeps C centrosymmetric).  ``dadd`` is added to the diagonal of C
// before the split (the z table carries the mass term c_m this way): rows
// 1..p-1 get dadd, the shared rows 0 and p get dadd/2 each, so a shared node,
// which sums row 0 of its element and row p of the element below, gets dadd
// once.
template <typename T, int P>
inline void build_eotab(const SemGeom& g, int d, const double (&rowmul)[P + 1], EOTab<T, P>& t,
                        double dadd = 0.0) {
  using TL = SemTile<P>;
  constexpr int H = TL::H;
  double Cm[P + 1][P + 1];
  for (int a = 0; a <= P; ++a)
    for (int l = 0; l <= P; ++l)
      Cm[a][l] = rowmul[a] * (g.C[d][a][l] + ((a == l) ? ((a == 0 || a == P) ? 0.5 * dadd : dadd) : 0.0));
  for (int a = 0; a < TL::HE; ++a) {
    const int aa = (a < H) ? a : P / 2;
    for (int l = 0; l < H; ++l) {
      t.ce[a][l] = (T)(0.5 * (Cm[aa][l] + Cm[aa][P - l]));
      if (a < H) t.co[a][l] = (T)(0.5 * (Cm[aa][l] - Cm[aa][P - l]));
    }
    if constexpr (TL::MID) t.cm[a] = (T)Cm[aa][P / 2];
  }
  if constexpr (!TL::MID) t.cm[0] = (T)0;
  for (int l = 0; l <= P; ++l) t.crow[l] = (T)Cm[P][l];
}

// The operator's SemTabs (host).
template <typename T, int P>
inline void sem_tables(const SemGeom& g, SemTabs<T, P>& tb) {
  double wz[P + 1], one[P + 1];
  for (int a = 0; a < P; ++a) wz[a] = g.wl[a];
  wz[P] = g.wl[0];
  for (int a = 0; a <= P; ++a) one[a] = 1.0;
  build_eotab<T, P>(g, 2, wz, tb.t[0], g.cm);
  build_eotab<T, P>(g, 0, one, tb.t[1]);
  build_eotab<T, P>(g, 1, one, tb.t[2]);
  for (int a = 0; a <= P; ++a) tb.w[a] = (T)g.wl[a];
}

// cp.async of one element, zero-filled when !valid (nothing is read then).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst_smem, const T* src, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst_smem);
  const int sz = valid ? (int)sizeof(T) : 0;
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(saddr), "l"(src), "r"(sz) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(saddr), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One work item: the CTA's element-aligned xy tile (bxi, byi) over element
// layers [e0, e1) of one mesh.  Adds this item's reduction terms to red[].
// Used by k_sem (one item per CTA) and by the persistent batched kernel.
template <typename T, int P, int MODE, bool SMEM>
__device__ __forceinline__ void sem_item(const SemGeom& g, const SemTabs<T, P>& tb, const SemArgs<T>& a, int bxi,
                                         int byi, int e0, int e1, const T* beta_s, const int* first_s, T (&red)[3],
                                         const int* skip_s = nullptr, bool lead_sync = true) {
  // tb: the operator's coefficients -- a kernel parameter (SMEM = false) or a
  // shared-memory copy the caller made and published with a barrier (SMEM).
  // beta_s, first_s: shared-memory scalars of the PCG step (MODE 1), published
  // by a barrier before the call and read at each use (held in registers they
  // cost the kernels more: 1.5 us per FP64 and FP32 step, measured).
  // skip_s: shared flag written before the call (the set-up barrier publishes
  // it); the item returns at once when it is set.  lead_sync = false: no earlier
  // item used this CTA's shared memory (k_sem), so the leading barrier is omitted.
  using TL = SemTile<P>;
  constexpr int TX = TL::TX, TY = TL::TY, PY = TL::PY, NPL = TL::NPL;
  constexpr int PXW = TL::PX;                    // staged row width
  constexpr int PX = TL::template pitch<T>();    // its pitch in shared memory
  constexpr int TEX = TL::TEX, TEY = TL::TEY, NT = TL::NTHREADS;
  constexpr int PLANE = PX * PY;
  constexpr int STAGED = PXW * PY;               // staged elements per plane
  constexpr int K = (STAGED + NT - 1) / NT;      // staged elements per thread per plane
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* S = reinterpret_cast<T*>(smem_raw);         // NPL ring slots of PY x PX
  constexpr bool TWO_W = TL::template two_w<T>();
  T* Wb = S + (size_t)NPL * PLANE;               // P planes of TY x TX (x results)
  T* Wy = TWO_W ? Wb + (size_t)P * TY * TX : Wb; // y results (same buffer for FP64)

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + TX * ty;
  if (lead_sync) __syncthreads();                // shared memory of a previous item is free
  if (skip_s && *skip_s) return;

  const int x0 = bxi * TX, y0 = byi * TY;
  // node indices: 32-bit for FP32 (n < 2^31; fewer address instructions,
  // 62.1 against 66.5 us for y = A x on 32^3), 64-bit for FP64 (whose register
  // allocation spills with the 32-bit form)
  using Idx = typename std::conditional<sizeof(T) == 4, int, size_t>::type;
  const Idx nxy = (Idx)g.nx * g.ny;

  // per-thread staging offsets of the padded plane (same for every plane)
  int soff[K], sdst[K];
  bool sval[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int i = tid + k * NT;
    const int py = i / PXW, px = i - py * PXW;
    const int gxk = x0 - P + px, gyk = y0 - P + py;
    sval[k] = (i < STAGED) && gxk > 0 && gyk > 0 && gxk < g.nx - 1 && gyk < g.ny - 1;
    soff[k] = sval[k] ? gxk + g.nx * gyk : 0;
    sdst[k] = py * PX + px;
  }
  auto stage_plane = [&](int gz) {
    T* plane = S + (size_t)(gz % NPL) * PLANE;
    const bool zok = gz > 0 && gz < g.nz - 1;
    const T* base = a.x + (zok ? (Idx)gz * nxy : 0);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = tid + k * NT;
      if (i < STAGED) cp_async_elem(plane + sdst[k], base + soff[k], zok && sval[k]);
    }
  };


  const int gx = x0 + tx, gy = y0 + ty;
  const int ia = tx % P, ib = ty % P;
  const bool col_in = (gx < g.nx - 1) && (gy < g.ny - 1);
  const bool col_int = col_in && gx > 0 && gy > 0;
  const T wxy = tb.w[ia] * tb.w[ib];
  const Idx colbase = (Idx)gx + (Idx)g.nx * gy;

  // prologue: stage the first layer (all p+1 planes)
  if (e0 < e1) {
    for (int pl = 0; pl <= P; ++pl) stage_plane(e0 * P + pl);
    cp_async_commit();
  }

  // FP64 over a single element layer: the p ring slots that no later layer
  // needs take this layer's epilogue operands of the owned nodes -- PCG step:
  // old q and p; residual: b and 1/diag -- (slot of plane c: the first at
  // [tid], the second at [NT + tid]), copied asynchronously while the line
  // products run (the FP32 kernel prefetches them into registers).
  constexpr bool PREF = sizeof(T) == 4;          // FP64: registers are too tight
  constexpr bool SPF_FITS = 2 * NT <= PLANE;     // a slot holds one plane's two operands
  const bool spf = SPF_FITS && !PREF && e1 == e0 + 1 && ((MODE == 1 && !*first_s) || MODE == 2);
  auto pq_slot = [&](int c) { return (e0 * P + P + 1 + c) % NPL; };
  if (spf) {
    const T* src0 = MODE == 1 ? a.out : a.aux;
    const T* src1 = MODE == 1 ? a.out2 : a.invd;
    const bool two = MODE == 1 || !a.final_pass;   // the true-residual pass reads b only
#pragma unroll
    for (int c = 0; c < P; ++c) {
      const Idx idx = colbase + nxy * (Idx)(e0 * P + c);
      T* sl = S + (size_t)pq_slot(c) * PLANE;
      cp_async_elem(sl + tid, src0 + (col_in ? idx : 0), col_in);
      if (two) cp_async_elem(sl + NT + tid, src1 + (col_in ? idx : 0), col_in);
    }
    cp_async_commit();
  }

  // z-carry from the element layer below the chunk (row p on its line)
  T carry = (T)0;
  if (e0 > 0 && col_int) {
    T ub[P + 1];
#pragma unroll
    for (int l = 0; l <= P; ++l) {
      const int gz = (e0 - 1) * P + l;
      ub[l] = (gz > 0) ? a.x[colbase + nxy * (Idx)gz] : (T)0;
    }
    carry = row_dot<T, P>(ub, tb.t[0]);
  }

  // x / y item coordinates (one item per thread per phase)
  const int xi_e = tid % TEX, xi_r = (tid / TEX) % TY, xi_c = tid / (TEX * TY);
  const int yi_e = tid % TEY, yi_r = (tid / TEY) % TX, yi_c = tid / (TEY * TX);

  for (int e = e0; e < e1; ++e) {
    // ---- prefetch the next layer's p new planes, then wait for this layer's
    if (e + 1 < e1) {
      for (int pl = 1; pl <= P; ++pl) stage_plane((e + 1) * P + pl);
      cp_async_commit();
      cp_async_wait<1>();
    } else if (spf) {
      cp_async_wait<1>();                        // the planes; q and p may still be in flight
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();

    // ring slot of plane e*P + l is slot0 + l (mod NPL)
    const int slot0 = (e * P) % NPL;
    auto slot_of = [&](int l) { int sl = slot0 + l; return sl >= NPL ? sl - NPL : sl; };

    // ---- z: own column in registers
    T u[P + 1], acc[P];
#pragma unroll
    for (int l = 0; l <= P; ++l)
      u[l] = S[slot_of(l) * PLANE + (ty + P) * PX + (tx + P)];
    {
      T o[P + 1];
      line_eo<T, P, false, SMEM>(u, u, tb.t[0], o);
#pragma unroll
      for (int c = 0; c < P; ++c) acc[c] = o[c];   // includes c_m u (folded into the z tables)
      acc[0] += carry;
      carry = o[P];
    }

    // epilogue operands of this layer's owned nodes (FP32), loaded before the x
    // and y contractions to overlap their latency with both (PCG step on 32^3:
    // 95.3 us; issued between x and y, 97.0 us; without the prefetch, 171 us)
    T ea[P], eb[P];
    if (PREF && (MODE == 1 || MODE == 2)) {
      const Idx lidx0 = colbase + nxy * (Idx)(e * P);
#pragma unroll
      for (int c = 0; c < P; ++c) {
        const Idx idx = lidx0 + nxy * (Idx)c;
        const bool ok = col_in && (MODE == 2 ? (col_int && e * P + c > 0) : !*first_s);
        ea[c] = ok ? (MODE == 1 ? a.out[idx] : a.aux[idx]) : (T)0;
        eb[c] = (ok && (MODE == 1 || !a.final_pass)) ? (MODE == 1 ? a.out2[idx] : a.invd[idx]) : (T)0;
      }
    }

    // ---- x: item (plane c, row, element) -> work buffer
    {
      const T* row = S + slot_of(xi_c) * PLANE + (xi_r + P) * PX + xi_e * P;
      T ul[P + 1], ue[P + 1], o[P + 1];
#pragma unroll
      for (int l = 0; l <= P; ++l) { ul[l] = row[l]; ue[l] = row[P + l]; }
      line_eo<T, P, true, SMEM>(ue, ul, tb.t[1], o);
      T* w = Wb + ((size_t)xi_c * TY + xi_r) * TX + xi_e * P;
#pragma unroll
      for (int c = 0; c < P; ++c) w[c] = o[c];
    }
    if constexpr (!TWO_W) __syncthreads();      // x results visible to the y items

    const Idx lidx = colbase + nxy * (Idx)(e * P);   // this layer's first owned node

    // ---- y: item (plane c, column, element) -> work buffer
    {
      const T* col = S + slot_of(yi_c) * PLANE + (yi_e * P) * PX + (yi_r + P);
      T ul[P + 1], ue[P + 1], o[P + 1];
#pragma unroll
      for (int l = 0; l <= P; ++l) { ul[l] = col[(size_t)l * PX]; ue[l] = col[(size_t)(P + l) * PX]; }
      line_eo<T, P, true, SMEM>(ue, ul, tb.t[2], o);
      T* w = Wy + ((size_t)yi_c * TY + yi_e * P) * TX + yi_r;
      if constexpr (TWO_W) {
#pragma unroll
        for (int c = 0; c < P; ++c) w[(size_t)c * TX] = o[c];
      } else {                                   // one buffer: add to the node's x result
#pragma unroll
        for (int c = 0; c < P; ++c) w[(size_t)c * TX] += o[c];
      }
    }
    __syncthreads();
    if constexpr (TWO_W) {   // x results of plane c carry the plane's weight W_c
#pragma unroll
      for (int c = 0; c < P; ++c) acc[c] = fma(tb.w[c], Wb[((size_t)c * TY + ty) * TX + tx], acc[c]);
    }

    // ---- combine, weights, epilogue
    if (spf) cp_async_wait<0>();                 // this thread's own operand copies
#pragma unroll
    for (int c = 0; c < P; ++c) {
      const int gz = e * P + c;
      const T v = fma(tb.w[c], Wy[((size_t)c * TY + ty) * TX + tx], acc[c]);   // (x +) y results x W_c
      const bool inside = col_int && gz > 0;
      const T yv = inside ? wxy * v : (T)0;
      if (col_in) {
        const Idx idx = lidx + nxy * (Idx)c;
        if (MODE == 0) {
          a.out[idx] = yv;
        } else if (MODE == 1) {
          T qv = yv, pv = u[c];
          if (!*first_s) {
            const T beta = *beta_s;
            const T* sl = S + (size_t)pq_slot(c) * PLANE;
            qv += beta * (PREF ? ea[c] : (spf ? sl[tid] : a.out[idx]));
            pv += beta * (PREF ? eb[c] : (spf ? sl[NT + tid] : a.out2[idx]));
          }
          a.out[idx] = qv;
          a.out2[idx] = pv;
          red[0] += pv * qv;
        } else {
          const T* sl = S + (size_t)pq_slot(c) * PLANE;
          const T bv = inside ? (PREF ? ea[c] : (spf ? sl[tid] : a.aux[idx])) : (T)0;
          const T rv = inside ? bv - yv : (T)0;
          a.out[idx] = rv;
          if (!a.final_pass) {
            const T zv = rv * (PREF ? eb[c] : (spf ? sl[NT + tid] : a.invd[idx]));
            a.out2[idx] = zv;
            red[1] += rv * zv;
          }
          red[0] += rv * rv;
          red[2] += bv * bv;
        }
      }
    }
  }

  // ---- upper Dirichlet faces (index n-1) inside this CTA's region: write 0.
  // The CTA covers x in [x0, xe), y in [y0, ye), z in [z0, ze) where the end is
  // extended to n when the CTA is the last one along that axis.
  {
    const bool lastx = (x0 + TX >= g.nx - 1), lasty = (y0 + TY >= g.ny - 1);
    const bool lastz = (e1 == g.ez);
    if (lastx || lasty || lastz) {
      const int xe = lastx ? g.nx : min(x0 + TX, g.nx), ye = lasty ? g.ny : min(y0 + TY, g.ny);
      const int z0 = e0 * P, ze = lastz ? g.nz : e1 * P;
      const int wx = xe - x0, wy = ye - y0, wz = ze - z0;
      auto zero_at = [&](int px, int py, int pz) {
        const Idx idx = (Idx)px + (Idx)g.nx * py + nxy * (Idx)pz;
        a.out[idx] = (T)0;
        if (MODE == 1 || (MODE == 2 && !a.final_pass)) a.out2[idx] = (T)0;
      };
      if (lastx)   // face x = nx-1
        for (int i = tid; i < wy * wz; i += NT) zero_at(g.nx - 1, y0 + i % wy, z0 + i / wy);
      if (lasty)   // face y = ny-1
        for (int i = tid; i < wx * wz; i += NT) zero_at(x0 + i % wx, g.ny - 1, z0 + i / wx);
      if (lastz)   // face z = nz-1
        for (int i = tid; i < wx * wy; i += NT) zero_at(x0 + i % wx, y0 + i / wx, g.nz - 1);
    }
  }

}

template <typename T, int P, int MODE>
__global__ void __launch_bounds__(SemTile<P>::NTHREADS, SemTile<P>::template minb<T>())
k_sem(const __grid_constant__ SemGeom g, const SemArgs<T> a, const __grid_constant__ SemTabs<T, P> tb) {
  __shared__ double sred[32 * 3];
  __shared__ int s_skip;
  __shared__ T s_beta;
  __shared__ int s_first;
  __shared__ double s_rz;     // MODE 1: r.z for alpha in the reduction's tail, read at the start
  const int tid = threadIdx.x + SemTile<P>::TX * threadIdx.y;
  if (tid == 0) {             // published by the table set-up barrier inside sem_item
    s_skip = (MODE == 1) ? a.st->done : 0;
    s_beta = (MODE == 1) ? (T)a.st->beta : (T)0;
    s_first = (MODE == 1) ? a.st->first : 1;
    if (MODE == 1) s_rz = a.st->rz;
  }
  T red[3] = {(T)0, (T)0, (T)0};
  // gridDim.z chunks of element layers, balanced: sizes differ by at most one
  const int e0 = (int)(((long long)blockIdx.z * g.ez) / gridDim.z);
  const int e1 = (int)(((long long)(blockIdx.z + 1) * g.ez) / gridDim.z);
  if constexpr (sizeof(T) == 8) {
    // FP64: the coefficients into shared memory (16-byte loads in the line
    // products); read from the parameter they would be hoisted into registers
    // the FP64 kernel does not have
    __shared__ SemTabs<T, P> s_tb;
    constexpr int NW = (int)(sizeof(SemTabs<T, P>) / sizeof(T));
    const T* src = reinterpret_cast<const T*>(&tb);
    T* dst = reinterpret_cast<T*>(&s_tb);
    for (int i = tid; i < NW; i += SemTile<P>::NTHREADS) dst[i] = src[i];
    __syncthreads();          // the tables and the shared scalars above
    sem_item<T, P, MODE, true>(g, s_tb, a, blockIdx.x, blockIdx.y, e0, e1, &s_beta, &s_first, red, &s_skip, false);
  } else {
    __syncthreads();          // the shared scalars above
    sem_item<T, P, MODE, false>(g, tb, a, blockIdx.x, blockIdx.y, e0, e1, &s_beta, &s_first, red, &s_skip, false);
  }
  if (MODE == 1 && s_skip) return;

  if (MODE == 1) {
    double v[1] = {(double)red[0]}, tot[1];
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
          st->alpha = s_rz / pq;
        }
      }
    }
  } else if (MODE == 2) {
    double v[3] = {(double)red[0], (double)red[1], (double)red[2]}, tot[3];
    if (grid_reduce_last<3>(v, a.partials, &a.st->counter[0], sred, tot)) {
      if (tid == 0) {
        PcgState* st = a.st;
        if (a.final_pass) {
          st->rr_true = tot[0];
          st->bb = tot[2];
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
