// sg_pcg.cu -- fused Jacobi-PCG (Sec. 5.3) with the stopping rules of Sec. 6.4.
//
// Per iteration two launches, all scalars kept on the device:
//   k_sem<MODE 1>:  w = A z; p = z + beta p, q = w + beta q (= A p by
//                   linearity; p = z, q = w first); p.q -> alpha = (r.z)/(p.q)
//   k_pcg_update:   x += alpha p, r -= alpha q, z = r / diag(A), r.r, r.z
//                   -> convergence test on ||r||, beta = (r.z)_new / (r.z)
// Applying A to z (which the update kernel has just written) instead of to the
// new p lets the operator stage a plain copy of one vector; p and q are then
// formed for owned nodes only.  The host launches a chunk of iterations and
// then reads the done flag once; kernels after convergence return at once.
// Vector traffic: 13 n words per iteration (5 in the operator kernel, 8 in
// the update).
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "sg_sem_launch.cuh"

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct PcgLayout {
  size_t state, partials, r, z, p, q, invd, total;
  int max_blocks;
};

// Grid of the update kernel.  FP64 (vec 2): 2 CTAs of 256 per SM -- its cost
// is FP64 instructions, and each block's r.r / r.z reduction adds FP64 work in
// proportion to the block count (8 CTAs per SM: 1.2 additions per node on the
// 16^3 p = 7 mesh, 2 per SM: 0.3; measured 3.32 -> 3.72 TB/s there).  (FP64
// with 3, 4, 6 CTAs per SM measured 23.8, 24.4, 27.4 us against 23.6 us.)
// FP32 (vec 4): up to 4 per SM and at least 4 elements per thread: with 8
// per SM a thread on a small mesh holds one element and spends its time in
// the launch and the block reduction (measured with compensated sums, same box:
// 16^3 p = 7 FP32 + replacement step 0.83 -> 0.78 ms, 32^3 122.4 -> 121.4 ms,
// four batched systems 51.8 -> 49.2 ms against 8 per SM).
int update_blocks(int64_t n, int vec) {
  int64_t nv = (n + vec - 1) / vec;
  int64_t b = vec == 2 ? (nv + 255) / 256 : (nv + 1023) / 1024;
  int64_t cap = (vec == 2 ? 2LL : 4LL) * sg_num_sms();
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

int sem_ctas(const SemGeom& g) {
  int tex = 1, tey = 1;
  switch (g.p) {
#define SG_CASE(P) case P: tex = SemTile<P>::TEX; tey = SemTile<P>::TEY; break;
    SG_CASE(1) SG_CASE(2) SG_CASE(3) SG_CASE(4) SG_CASE(5) SG_CASE(6) SG_CASE(7) SG_CASE(8)
#undef SG_CASE
  }
  // one layer per CTA: the most CTAs any layer count (sg_op_set_layers) gives,
  // so a workspace sized before the count changes still holds the partials
  return ((g.ex + tex - 1) / tex) * ((g.ey + tey - 1) / tey) * g.ez;
}

PcgLayout layout_for(sg_op_t op) {
  PcgLayout L{};
  const size_t es = op->dtype == SG_F64 ? 8 : 4;
  const size_t vb = align_up(es * (size_t)op->n);
  int mb = sem_ctas(op->g);
  int ub = update_blocks(op->n, op->dtype == SG_F64 ? 2 : 4);
  L.max_blocks = mb > ub ? mb : ub;
  size_t off = 0;
  L.state = off; off += align_up(sizeof(PcgState));
  L.partials = off; off += align_up(sizeof(double) * 4 * (size_t)L.max_blocks);
  L.r = off; off += vb;
  L.z = off; off += vb;
  L.p = off; off += vb;
  L.q = off; off += vb;
  L.invd = off; off += vb;
  L.total = off;
  return L;
}

// Tag of the inverse diagonal held in a workspace: derived from the operator's
// unique id, checked on the device so a workspace whose contents changed (or a
// fresh one) always gets the diagonal recomputed.
inline unsigned long long diag_tag(sg_op_t op) { return 0x5347494e56444941ull ^ (op->uid * 0x9e3779b97f4a7c15ull); }

struct PollBuf { int iter, done, status, pad; };

}  // namespace

template <typename T>
__global__ void k_mask_faces(T* v, int nx, int ny, int nz) {
  const size_t nxy = (size_t)nx * ny;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = t0; i < nx * ny; i += stride) {          // z faces
    v[i] = (T)0;
    v[(size_t)(nz - 1) * nxy + i] = (T)0;
  }
  for (int i = t0; i < nx * nz; i += stride) {          // y faces
    int xi = i % nx, zi = i / nx;
    v[(size_t)zi * nxy + xi] = (T)0;
    v[(size_t)zi * nxy + (size_t)(ny - 1) * nx + xi] = (T)0;
  }
  for (int i = t0; i < ny * nz; i += stride) {          // x faces
    int yi = i % ny, zi = i / ny;
    v[(size_t)zi * nxy + (size_t)yi * nx] = (T)0;
    v[(size_t)zi * nxy + (size_t)yi * nx + nx - 1] = (T)0;
  }
}

// 1/diag(A) into out unless the workspace already holds it for this operator.
template <typename T>
__global__ void k_inv_diag_cached(const SemGeom g, FastDiv dnx, FastDiv dnxy, int n, T* out,
                                  const PcgState* st, unsigned long long tag) {
  if (st->diag_tag == tag) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t k = dnxy.div((uint32_t)i);
    uint32_t rem = (uint32_t)i - k * dnxy.d;
    uint32_t j = dnx.div(rem);
    uint32_t ii = rem - j * dnx.d;
    double v = 1.0;
    if (ii > 0 && j > 0 && k > 0 && (int)ii < g.nx - 1 && (int)j < g.ny - 1 && (int)k < g.nz - 1) {
      int a = ii % g.p, b = j % g.p, c = k % g.p;
      v = g.wl[a] * g.wl[b] * g.wl[c] * (g.dg[0][a] + g.dg[1][b] + g.dg[2][c] + g.cm);
    }
    out[i] = (T)(1.0 / v);
  }
}

// The solve's small set-up in one launch: Dirichlet entries of x to 0
// (as k_mask_faces) and, by block 0, the tag of the diagonal just ensured and
// the state reset (as k_pcg_setup).  Runs after k_inv_diag_cached in stream order.
template <typename T>
__global__ void k_pcg_setup_all(T* x, int nx, int ny, int nz, PcgState* st, unsigned long long tag, double tol,
                                int maxit, int criterion) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->diag_tag = tag;
    st->rz = st->pq = st->rr = st->bb = st->rr0 = st->thr2 = 0.0;
    st->alpha = st->beta = st->rr_true = 0.0;
    st->iter = 0; st->done = 0; st->status = PCG_RUNNING; st->first = 1;
    st->maxit = maxit; st->criterion = criterion; st->tol = tol;
    st->xvec = x;
    for (int i = 0; i < 4; ++i) st->counter[i] = 0u;
  }
  const size_t nxy = (size_t)nx * ny;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = t0; i < nx * ny; i += stride) {          // z faces
    x[i] = (T)0;
    x[(size_t)(nz - 1) * nxy + i] = (T)0;
  }
  for (int i = t0; i < nx * nz; i += stride) {          // y faces
    int xi = i % nx, zi = i / nx;
    x[(size_t)zi * nxy + xi] = (T)0;
    x[(size_t)zi * nxy + (size_t)(ny - 1) * nx + xi] = (T)0;
  }
  for (int i = t0; i < ny * nz; i += stride) {          // x faces
    int yi = i % ny, zi = i / ny;
    x[(size_t)zi * nxy + (size_t)yi * nx] = (T)0;
    x[(size_t)zi * nxy + (size_t)yi * nx + nx - 1] = (T)0;
  }
}

__global__ void k_pcg_setup(PcgState* st, double tol, int maxit, int criterion, void* x) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    st->rz = st->pq = st->rr = st->bb = st->rr0 = st->thr2 = 0.0;
    st->alpha = st->beta = st->rr_true = 0.0;
    st->iter = 0; st->done = 0; st->status = PCG_RUNNING; st->first = 1;
    st->maxit = maxit; st->criterion = criterion; st->tol = tol;
    st->xvec = x;
    for (int i = 0; i < 4; ++i) st->counter[i] = 0u;
  }
}

template <typename T> struct Vec;
template <> struct Vec<double> { using V = double2; static constexpr int W = 2; };
template <> struct Vec<float> { using V = float4; static constexpr int W = 4; };

template <typename T>
__device__ __forceinline__ void upd1(T& x, T p, T& r, T q, T id, T& z, T al, T& rr, T& rz) {
  x += al * p;
  r -= al * q;
  z = r * id;
  rr += r * r;
  rz += r * z;
}

// x == NULL: the solution vector recorded in the state by k_pcg_setup (the
// form captured in the iteration graph).  use_cond: the launch is a node of the
// graph's WHILE body; the last block (or, once the solve is done, block 0)
// sets the loop condition to "not done".
template <typename T>
__global__ void __launch_bounds__(256)
k_pcg_update(T* __restrict__ x_arg, const T* __restrict__ p, T* __restrict__ r, const T* __restrict__ q,
             const T* __restrict__ invd, T* __restrict__ z, int n, PcgState* st, double* partials,
             cudaGraphConditionalHandle cond, int use_cond) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
  __shared__ int s_skip;
  __shared__ double s_alpha;
  __shared__ T* s_x;
  __shared__ double sred[64];
  // the state the reduction's tail needs, read at the start (no block of this
  // kernel changes it before the tail): no dependent loads in the serial tail
  __shared__ double s_rz, s_thr2;
  __shared__ int s_iter, s_maxit, s_strict;
  const int nv = n / W;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  // FP64: the first element's p, r, q and 1/diag loads go out before the state
  // is read and published (x's address comes from the state), so their latency
  // overlaps the state read at the start of this one-wave launch
  using VA = typename std::conditional<W == 2, V, char>::type;
  VA xa, pa, ra, qa, da;
  if constexpr (W == 2) {
    if (i < nv) {
      pa = reinterpret_cast<const V*>(p)[i]; ra = reinterpret_cast<V*>(r)[i];
      qa = reinterpret_cast<const V*>(q)[i]; da = reinterpret_cast<const V*>(invd)[i];
    }
  }
  if (threadIdx.x == 0) {
    s_skip = st->done; s_alpha = st->alpha; s_x = x_arg ? x_arg : static_cast<T*>(st->xvec);
    s_rz = st->rz; s_thr2 = st->thr2; s_iter = st->iter; s_maxit = st->maxit;
    s_strict = st->criterion != SG_STOP_REL_B;
  }
  __syncthreads();
  if (s_skip) {
    if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
    return;
  }
  T* __restrict__ x = s_x;
  const T al = (T)s_alpha;
  T rr = 0, rz = 0;
  // FP32: compensated (Kahan) per-thread sums of r.r and r.z -- their terms are
  // non-negative, and a plain FP32 running sum over tens of terms per thread
  // changes CG iteration counts (32^3 p = 7 Poisson, FP32 + replacement: 750
  // iterations at 37 terms per thread, 777 at 148)
  T crr = 0, crz = 0;
  auto kadd = [](T& sum, T& c, T v) { const T y = v - c; const T t = sum + y; c = (t - sum) - y; sum = t; };
  const int stride = gridDim.x * blockDim.x;
  auto step = [&](V& xv, const V& pv, V& rv, const V& qv, const V& dv, V& zv) {
    if constexpr (W == 4) {
      T r4 = 0, z4 = 0;                      // this element's four terms, then one compensated add
      upd1(xv.x, pv.x, rv.x, qv.x, dv.x, zv.x, al, r4, z4);
      upd1(xv.y, pv.y, rv.y, qv.y, dv.y, zv.y, al, r4, z4);
      upd1(xv.z, pv.z, rv.z, qv.z, dv.z, zv.z, al, r4, z4);
      upd1(xv.w, pv.w, rv.w, qv.w, dv.w, zv.w, al, r4, z4);
      kadd(rr, crr, r4);
      kadd(rz, crz, z4);
    } else {
      upd1(xv.x, pv.x, rv.x, qv.x, dv.x, zv.x, al, rr, rz);
      upd1(xv.y, pv.y, rv.y, qv.y, dv.y, zv.y, al, rr, rz);
    }
  };
  // FP64 (2 CTAs per SM, each thread ~9 grid-stride elements): software
  // pipelined -- the five loads of the next element are issued before this
  // element's FP64 work, so the loads of every warp stay in flight while the
  // FP64 pipe computes; FP32 runs a full wave and keeps its registers for
  // occupancy
  if constexpr (W == 2) {
    if (i < nv) xa = reinterpret_cast<V*>(x)[i];
    for (; i < nv; i += stride) {
      const int j = i + stride;
      V xb, pb, rb, qb, db;
      if (j < nv) {
        xb = reinterpret_cast<V*>(x)[j]; pb = reinterpret_cast<const V*>(p)[j];
        rb = reinterpret_cast<V*>(r)[j]; qb = reinterpret_cast<const V*>(q)[j];
        db = reinterpret_cast<const V*>(invd)[j];
      }
      V za;
      step(xa, pa, ra, qa, da, za);
      reinterpret_cast<V*>(x)[i] = xa;
      reinterpret_cast<V*>(r)[i] = ra;
      reinterpret_cast<V*>(z)[i] = za;
      xa = xb; pa = pb; ra = rb; qa = qb; da = db;
    }
  }
  for (; W == 4 && i < nv; i += stride) {
    V xv = reinterpret_cast<V*>(x)[i];
    V rv = reinterpret_cast<V*>(r)[i];
    V zv;
    step(xv, reinterpret_cast<const V*>(p)[i], rv, reinterpret_cast<const V*>(q)[i],
         reinterpret_cast<const V*>(invd)[i], zv);
    reinterpret_cast<V*>(x)[i] = xv;
    reinterpret_cast<V*>(r)[i] = rv;
    reinterpret_cast<V*>(z)[i] = zv;
  }
  for (int i = nv * W + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    T xs = x[i], rs = r[i], zs;
    upd1(xs, p[i], rs, q[i], invd[i], zs, al, rr, rz);
    x[i] = xs; r[i] = rs; z[i] = zs;
  }
  double v[2] = {(double)rr - (double)crr, (double)rz - (double)crz}, tot[2];
  if (grid_reduce_last<2>(v, partials, &st->counter[1], sred, tot)) {
    if (threadIdx.x == 0) {
      const int it = s_iter + 1;
      st->iter = it;
      st->rr = tot[0];
      const bool conv = s_strict ? (tot[0] < s_thr2) : (tot[0] <= s_thr2);
      int done = 0;
      if (!isfinite(tot[0]) || !isfinite(tot[1])) { st->status = PCG_BREAKDOWN; done = 1; }
      else if (conv) { st->status = PCG_CONVERGED; done = 1; }
      else {
        st->beta = tot[1] / s_rz;
        st->rz = tot[1];
        if (it >= s_maxit) { st->status = PCG_MAXIT; done = 1; }
      }
      if (done) st->done = 1;
      if (use_cond) cudaGraphSetConditional(cond, done ? 0u : 1u);
    }
  }
}

// Library-side kernel timing around a launch, compiled out for the
// allocation-free entry point (event creation allocates).
template <bool ON>
struct MaybeProf { MaybeProf(int, cudaStream_t) {} };
template <>
struct MaybeProf<true> { ProfScope ps; MaybeProf(int id, cudaStream_t s) : ps(id, s) {} };

// ---------------------------------------------------------------- device-driven iterations
// The iterations of a solve can run as one CUDA graph: a conditional WHILE node
// whose body is the operator step (k_sem MODE 1) followed by the update
// (k_pcg_update), which sets the loop condition to "not done" after every
// iteration.  No host poll and no per-iteration launch: the host enqueues the
// set-up kernels and one graph launch.  The graph references only the
// workspace (the solution vector is taken from the PCG state), so it is built
// once per (operator, workspace address) and cached on the operator.
namespace {
struct PcgGraphEntry { const void* ws; cudaGraphExec_t exec; };
struct PcgGraphCache {
  std::vector<PcgGraphEntry> entries;   // most recent last
  bool unavailable = false;             // graph construction failed once: use launches
  std::string why;
};
constexpr size_t kGraphCacheMax = 8;

PcgGraphCache* graph_cache(sg_op_t op) {
  if (!op->pcg_graphs) op->pcg_graphs = new PcgGraphCache();
  return static_cast<PcgGraphCache*>(op->pcg_graphs);
}

template <typename T>
int build_iteration_graph_ptrs(sg_op_t op, const PcgIterPtrs<T>& v, cudaGraphExec_t* out) {
  const int n = (int)op->n;
  int rc = sg_sem_prepare<T, 1>(op->g);
  if (rc) return rc;
  cudaGraph_t graph = nullptr, body = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraphConditionalHandle cond = 0;
  cudaGraphNode_t node;
  cudaGraphNodeParams cp = {};
  cudaError_t e = cudaGraphCreate(&graph, 0);
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  }
  if (e == cudaSuccess) {
    body = cp.conditional.phGraph_out[0];
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  }
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    SemArgs<T> a{};
    a.x = v.z; a.out = v.q; a.out2 = v.p;
    a.partials = v.partials; a.st = v.st;
    rc = sg_sem_launch<T, 1>(op->g, a, cs, 0);
    if (rc == SG_OK) {
      k_pcg_update<T><<<update_blocks(op->n, Vec<T>::W), 256, 0, cs>>>(v.x, v.p, v.r, v.q, v.invd, v.z, n, v.st,
                                                                    v.partials, cond, 1);
      e = cudaGetLastError();
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &captured);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess && rc == SG_OK) e = cudaGraphInstantiate(out, graph, 0);
  if (cs) cudaStreamDestroy(cs);
  if (graph) cudaGraphDestroy(graph);
  if (rc) return rc;
  if (e != cudaSuccess) return sg_fail(SG_ERR_CUDA, std::string("pcg iteration graph: ") + cudaGetErrorString(e));
  return SG_OK;
}

template <typename T>
int build_iteration_graph(sg_op_t op, unsigned char* ws, const PcgLayout& L, cudaGraphExec_t* out) {
  PcgIterPtrs<T> v{};
  v.st = reinterpret_cast<PcgState*>(ws + L.state);
  v.partials = reinterpret_cast<double*>(ws + L.partials);
  v.r = reinterpret_cast<T*>(ws + L.r);
  v.z = reinterpret_cast<T*>(ws + L.z);
  v.p = reinterpret_cast<T*>(ws + L.p);
  v.q = reinterpret_cast<T*>(ws + L.q);
  v.invd = reinterpret_cast<T*>(ws + L.invd);
  v.x = nullptr;                         // the solution vector recorded in the state
  return build_iteration_graph_ptrs<T>(op, v, out);
}

// The cached graph for (op, ws), built on first use; NULL (and the reason in
// the cache) when graphs cannot be built on this device.
template <typename T>
cudaGraphExec_t iteration_graph(sg_op_t op, unsigned char* ws, const PcgLayout& L) {
  PcgGraphCache* c = graph_cache(op);
  if (c->unavailable) return nullptr;
  for (size_t i = 0; i < c->entries.size(); ++i) {
    if (c->entries[i].ws == ws) {
      PcgGraphEntry hit = c->entries[i];
      c->entries.erase(c->entries.begin() + (long)i);
      c->entries.push_back(hit);
      return hit.exec;
    }
  }
  cudaGraphExec_t exec = nullptr;
  if (build_iteration_graph<T>(op, ws, L, &exec) != SG_OK) {
    c->unavailable = true;
    c->why = sg_last_error();
    cudaGetLastError();
    return nullptr;
  }
  if (c->entries.size() >= kGraphCacheMax) {
    cudaGraphExecDestroy(c->entries.front().exec);   // freed after any launch in flight completes
    c->entries.erase(c->entries.begin());
  }
  c->entries.push_back({ws, exec});
  return exec;
}
}  // namespace

// Iteration graph over explicit vectors (the batched solver's single-system
// tail, sg_batch.cu): x is updated in place, the loop runs while st->done == 0.
int sg_pcg_iteration_graph_f32(sg_op_t op, const PcgIterPtrs<float>& v, cudaGraphExec_t* out) {
  return build_iteration_graph_ptrs<float>(op, v, out);
}

void sg_pcg_release(sg_op_s* op) {
  if (!op || !op->pcg_graphs) return;
  PcgGraphCache* c = static_cast<PcgGraphCache*>(op->pcg_graphs);
  for (auto& en : c->entries) cudaGraphExecDestroy(en.exec);
  delete c;
  op->pcg_graphs = nullptr;
}

// Relative tolerance of one inner solve of refinement (ir_inner_tol).
__host__ __device__ inline double ir_seg_tol(double inner_tol, double tol, double rel) {
  double t = 0.5 * tol / rel;
  if (t < inner_tol) t = inner_tol;
  return t < 0.1 ? t : (inner_tol > 0.1 ? inner_tol : 0.1);
}

// First segment of residual replacement, enqueued before the host has seen the
// FP64 residual: the segment's tolerance from that residual (rr_true, bb in
// ref, written by the residual pass before this launch).  When the residual
// already meets tol, or is not finite, the segment's iteration limit becomes 0
// (the set-up pass then ends it without work) and pad[0] records the skip.
__global__ void k_ru_first_tol(const PcgState* ref, PcgState* st, double delta, double tol) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double rel = ref->bb > 0 ? sqrt(ref->rr_true / ref->bb) : sqrt(ref->rr_true);
  const bool skip = !(rel > tol);            // also when rel is not finite
  st->tol = skip ? 0.1 : ir_seg_tol(delta, tol, rel);
  if (skip) st->maxit = 0;
  st->pad[0] = skip ? 1 : 0;
}

// Set-up of a solve on the stream: 1/diag(A) (unless cached), Dirichlet
// entries of x to 0, state reset, r = b - A x, z = r / diag(A), r.r, r.z, b.b.
// tol_ref: the tolerance comes from a residual on the device (k_ru_first_tol).
template <typename T>
static int pcg_start(sg_op_t op, const T* b, T* x, double tol, int maxit, int criterion, unsigned char* ws,
                     const PcgLayout& L, cudaStream_t s, const PcgState* tol_ref = nullptr, double ref_delta = 0.0,
                     double ref_tol = 0.0) {
  PcgState* st = reinterpret_cast<PcgState*>(ws + L.state);
  T* invd = reinterpret_cast<T*>(ws + L.invd);
  const int n = (int)op->n;
  const SemGeom& g = op->g;
  const unsigned long long tag = diag_tag(op);
  // one wave (2 CTAs per SM): when the workspace holds the diagonal already,
  // every CTA only reads the tag and returns
  int blocks = (n + 255) / 256;
  if (blocks > 2 * sg_num_sms()) blocks = 2 * sg_num_sms();
  k_inv_diag_cached<T><<<blocks, 256, 0, s>>>(g, op->div_nx, op->div_nxy, n, invd, st, tag);
  SG_LAUNCH_CHECK("k_inv_diag_cached");
  k_pcg_setup_all<T><<<64, 256, 0, s>>>(x, g.nx, g.ny, g.nz, st, tag, tol, maxit, criterion);
  SG_LAUNCH_CHECK("k_pcg_setup_all");
  if (tol_ref) {
    k_ru_first_tol<<<1, 32, 0, s>>>(tol_ref, st, ref_delta, ref_tol);
    SG_LAUNCH_CHECK("k_ru_first_tol");
  }
  SemArgs<T> a{};
  a.x = x; a.aux = b; a.invd = invd; a.out = reinterpret_cast<T*>(ws + L.r); a.out2 = reinterpret_cast<T*>(ws + L.z);
  a.partials = reinterpret_cast<double*>(ws + L.partials); a.st = st; a.final_pass = 0;
  return sg_sem_launch<T, 2>(g, a, s, 0);
}

// Iterations by host launches: chunks of (operator step, update) pairs, the
// done flag read after each chunk.  The first chunk is sized from the previous
// solve with this operator, so a sequence of similar solves usually needs one
// poll; launches beyond convergence return at once.  Used when kernels are
// timed one by one (sg_profile_enable), by the allocation-free entry point,
// and where graphs cannot be built.
template <typename T, bool NOALLOC>
static int pcg_iterate_launches(sg_op_t op, T* x, int maxit, unsigned char* ws, const PcgLayout& L, cudaStream_t s) {
  PcgState* st = reinterpret_cast<PcgState*>(ws + L.state);
  double* partials = reinterpret_cast<double*>(ws + L.partials);
  T* r = reinterpret_cast<T*>(ws + L.r);
  T* z = reinterpret_cast<T*>(ws + L.z);
  T* p = reinterpret_cast<T*>(ws + L.p);
  T* q = reinterpret_cast<T*>(ws + L.q);
  T* invd = reinterpret_cast<T*>(ws + L.invd);
  const int n = (int)op->n;
  const int ub = update_blocks(op->n, Vec<T>::W);
  PollBuf local_poll{};      // pageable host memory: no pinned allocation
  PollBuf* poll = &local_poll;
  if constexpr (!NOALLOC) {
    static thread_local PollBuf* pinned = nullptr;
    if (!pinned) SG_CUDA_TRY(cudaHostAlloc((void**)&pinned, sizeof(PollBuf), cudaHostAllocDefault));
    poll = pinned;
  }
  int launched = 0;
  int chunk = op->last_iters > 0 ? (op->last_iters < 64 ? op->last_iters + 1 : 64) : 4;
  bool first_chunk = true;
  while (true) {
    if (!first_chunk) {
      SG_CUDA_TRY(cudaMemcpyAsync(poll, &st->iter, sizeof(int) * 3, cudaMemcpyDeviceToHost, s));
      SG_CUDA_TRY(cudaStreamSynchronize(s));
      if (poll->done) break;
    }
    first_chunk = false;
    if (launched >= maxit) break;            // the device sets done at maxit
    const int k = (chunk < maxit - launched) ? chunk : (maxit - launched);
    for (int i = 0; i < k; ++i) {
      {
        MaybeProf<!NOALLOC> ps(PROF_PCG_APPLY, s);
        SemArgs<T> a{};
        a.x = z; a.out = q; a.out2 = p;
        a.partials = partials; a.st = st;
        int rc = sg_sem_launch<T, 1>(op->g, a, s, 0);
        if (rc) return rc;
      }
      {
        MaybeProf<!NOALLOC> ps(PROF_PCG_UPDATE, s);
        k_pcg_update<T><<<ub, 256, 0, s>>>(x, p, r, q, invd, z, n, st, partials, 0, 0);
        SG_LAUNCH_CHECK("k_pcg_update");
      }
    }
    launched += k;
    chunk = (chunk < 8) ? 8 : (chunk < 16 ? 16 : chunk);
  }
  return SG_OK;
}

// Outcome of the solve in this workspace (synchronises): iteration count,
// status, and with relres the true relative residual ||b - A x|| / ||b||
// (one more operator pass).
template <typename T>
static int pcg_finish(sg_op_t op, const T* b, T* x, unsigned char* ws, const PcgLayout& L, int* iters,
                      double* relres, cudaStream_t s, bool count_graph_launches) {
  PcgState* st = reinterpret_cast<PcgState*>(ws + L.state);
  if (relres) {
    SemArgs<T> a{};
    a.x = x; a.aux = b; a.invd = reinterpret_cast<T*>(ws + L.invd);
    a.out = reinterpret_cast<T*>(ws + L.r); a.out2 = reinterpret_cast<T*>(ws + L.z);
    a.partials = reinterpret_cast<double*>(ws + L.partials); a.st = st; a.final_pass = 1;
    int rc = sg_sem_launch<T, 2>(op->g, a, s, 0);
    if (rc) return rc;
  }
  PcgState hs;
  SG_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  SG_CUDA_TRY(cudaStreamSynchronize(s));
  if (count_graph_launches) sg_count_launches(2 * (hs.iter > 0 ? hs.iter : 1));   // body kernels the graph ran
  if (iters) *iters = hs.iter;
  op->last_iters = hs.iter;
  if (relres) *relres = hs.bb > 0 ? sqrt(hs.rr_true / hs.bb) : sqrt(hs.rr_true);
  if (hs.status == PCG_BREAKDOWN) return sg_fail(SG_ERR_BREAKDOWN, "pcg: breakdown (p^T A p <= 0 or non-finite value)");
  if (hs.status == PCG_MAXIT || hs.status == PCG_RUNNING) {
    sg_set_error("pcg: maximum iteration count reached");
    return SG_NOT_CONVERGED;
  }
  return SG_OK;
}

template <typename T, bool NOALLOC = false>
static int pcg_run(sg_op_t op, const T* b, T* x, double tol, int maxit, int criterion,
                   unsigned char* ws, const PcgLayout& L, int* iters, double* relres, cudaStream_t s) {
  int rc = pcg_start<T>(op, b, x, tol, maxit, criterion, ws, L, s);
  if (rc) return rc;
  cudaGraphExec_t exec = nullptr;
  if (!NOALLOC && !sg_profiling_on()) exec = iteration_graph<T>(op, ws, L);
  if (exec) {
    SG_CUDA_TRY(cudaGraphLaunch(exec, s));
  } else {
    rc = pcg_iterate_launches<T, NOALLOC>(op, x, maxit, ws, L, s);
    if (rc) return rc;
  }
  return pcg_finish<T>(op, b, x, ws, L, iters, relres, s, exec != nullptr);
}

extern "C" int sg_residual_norm(sg_op_t op, const void* b, const void* x, void* workspace, double* relres,
                                void* stream) {
  if (!op || !b || !x || !workspace || !relres) return sg_fail(SG_ERR_INVALID, "residual_norm: NULL argument");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return sg_fail(SG_ERR_INVALID, "residual_norm: workspace must be 256-byte aligned");
  PcgLayout L = layout_for(op);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  PcgState* st = reinterpret_cast<PcgState*>(ws + L.state);
  cudaStream_t s = as_stream(stream);
  k_pcg_setup<<<1, 32, 0, s>>>(st, 1.0, 0, SG_STOP_REL_B, nullptr);
  SG_LAUNCH_CHECK("k_pcg_setup");
  int rc;
  if (op->dtype == SG_F64) {
    SemArgs<double> a{};
    a.x = static_cast<const double*>(x); a.aux = static_cast<const double*>(b);
    a.out = reinterpret_cast<double*>(ws + L.r);
    a.partials = reinterpret_cast<double*>(ws + L.partials); a.st = st; a.final_pass = 1;
    rc = sg_sem_launch<double, 2>(op->g, a, s, 0);
  } else {
    SemArgs<float> a{};
    a.x = static_cast<const float*>(x); a.aux = static_cast<const float*>(b);
    a.out = reinterpret_cast<float*>(ws + L.r);
    a.partials = reinterpret_cast<double*>(ws + L.partials); a.st = st; a.final_pass = 1;
    rc = sg_sem_launch<float, 2>(op->g, a, s, 0);
  }
  if (rc) return rc;
  PcgState hs;
  SG_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
  SG_CUDA_TRY(cudaStreamSynchronize(s));
  *relres = hs.bb > 0 ? sqrt(hs.rr_true / hs.bb) : sqrt(hs.rr_true);
  return SG_OK;
}

static int pcg_check_args(sg_op_t op, const void* b, void* x, double tol, int maxit, int criterion, void* workspace,
                          const char* who) {
  const std::string w(who);
  if (!op || !b || !x || !workspace) return sg_fail(SG_ERR_INVALID, w + ": NULL argument");
  if (!(tol > 0.0)) return sg_fail(SG_ERR_INVALID, w + ": tol must be > 0");
  if (maxit < 0) return sg_fail(SG_ERR_INVALID, w + ": maxit must be >= 0");
  if (criterion < 0 || criterion > 2) return sg_fail(SG_ERR_INVALID, w + ": unknown criterion");
  if (!aligned16(b) || !aligned16(x)) return sg_fail(SG_ERR_INVALID, w + ": vectors must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return sg_fail(SG_ERR_INVALID, w + ": workspace must be 256-byte aligned");
  if (b == x) return sg_fail(SG_ERR_INVALID, w + ": b and x must not alias");
  return SG_OK;
}

extern "C" size_t sg_pcg_workspace_bytes(sg_op_t op) {
  if (!op) return 0;
  return layout_for(op).total;
}

extern "C" int sg_pcg_solve(sg_op_t op, const void* b, void* x, double tol, int maxit, int criterion,
                            void* workspace, int* iters, double* relres, void* stream) {
  int rc = pcg_check_args(op, b, x, tol, maxit, criterion, workspace, "pcg_solve");
  if (rc) return rc;
  PcgLayout L = layout_for(op);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  cudaStream_t s = as_stream(stream);
  if (op->dtype == SG_F64)
    return pcg_run<double>(op, static_cast<const double*>(b), static_cast<double*>(x), tol, maxit,
                           criterion, ws, L, iters, relres, s);
  return pcg_run<float>(op, static_cast<const float*>(b), static_cast<float*>(x), tol, maxit,
                        criterion, ws, L, iters, relres, s);
}

template <typename T>
static int pcg_enqueue(sg_op_t op, const T* b, T* x, double tol, int maxit, int criterion, unsigned char* ws,
                       const PcgLayout& L, cudaStream_t s) {
  cudaGraphExec_t exec = iteration_graph<T>(op, ws, L);
  if (!exec)
    return sg_fail(SG_ERR_CUDA, "pcg_solve_async: iteration graph unavailable: " +
                                static_cast<PcgGraphCache*>(op->pcg_graphs)->why);
  int rc = pcg_start<T>(op, b, x, tol, maxit, criterion, ws, L, s);
  if (rc) return rc;
  SG_CUDA_TRY(cudaGraphLaunch(exec, s));
  return SG_OK;
}

extern "C" int sg_pcg_solve_async(sg_op_t op, const void* b, void* x, double tol, int maxit, int criterion,
                                  void* workspace, void* stream) {
  int rc = pcg_check_args(op, b, x, tol, maxit, criterion, workspace, "pcg_solve_async");
  if (rc) return rc;
  PcgLayout L = layout_for(op);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  cudaStream_t s = as_stream(stream);
  if (op->dtype == SG_F64)
    return pcg_enqueue<double>(op, static_cast<const double*>(b), static_cast<double*>(x), tol, maxit, criterion,
                               ws, L, s);
  return pcg_enqueue<float>(op, static_cast<const float*>(b), static_cast<float*>(x), tol, maxit, criterion, ws, L, s);
}

extern "C" int sg_pcg_result(sg_op_t op, void* workspace, int* iters, void* stream) {
  if (!op || !workspace) return sg_fail(SG_ERR_INVALID, "pcg_result: NULL argument");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return sg_fail(SG_ERR_INVALID, "pcg_result: workspace must be 256-byte aligned");
  PcgLayout L = layout_for(op);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  cudaStream_t s = as_stream(stream);
  if (op->dtype == SG_F64)
    return pcg_finish<double>(op, nullptr, nullptr, ws, L, iters, nullptr, s, true);
  return pcg_finish<float>(op, nullptr, nullptr, ws, L, iters, nullptr, s, true);
}

// ---------------------------------------------------------------- allocation-free PCG
// Scratch for sg_pcg_solve_noalloc: a file-scope device array, so the call needs
// no workspace from the caller and allocates nothing.  Every device that loads
// the library holds these SG_NOALLOC_SCRATCH_BYTES until the process exits.
static __device__ __align__(256) unsigned char g_pcg_scratch[SG_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mu;
void* g_scratch_addr[64] = {nullptr};   // device address of g_pcg_scratch, per device
}

extern "C" int sg_pcg_solve_noalloc(sg_op_t op, const void* b, void* x, double tol, int maxit,
                                    int criterion, int* iters, double* relres, void* stream) {
  if (!op || !b || !x) return sg_fail(SG_ERR_INVALID, "pcg_solve_noalloc: NULL argument");
  if (op->n > SG_NOALLOC_MAX_NODES)
    return sg_fail(SG_ERR_INVALID, "pcg_solve_noalloc: operator has " + std::to_string(op->n) +
                                   " nodes, above the maximum of " + std::to_string(SG_NOALLOC_MAX_NODES));
  if (!(tol > 0.0)) return sg_fail(SG_ERR_INVALID, "pcg_solve_noalloc: tol must be > 0");
  if (maxit < 0) return sg_fail(SG_ERR_INVALID, "pcg_solve_noalloc: maxit must be >= 0");
  if (criterion < 0 || criterion > 2) return sg_fail(SG_ERR_INVALID, "pcg_solve_noalloc: unknown criterion");
  if (!aligned16(b) || !aligned16(x)) return sg_fail(SG_ERR_INVALID, "pcg_solve_noalloc: vectors must be 16-byte aligned");
  if (b == x) return sg_fail(SG_ERR_INVALID, "pcg_solve_noalloc: b and x must not alias");
  PcgLayout L = layout_for(op);
  if (L.total > SG_NOALLOC_SCRATCH_BYTES)
    return sg_fail(SG_ERR_INVALID, "pcg_solve_noalloc: scratch of " + std::to_string(L.total) +
                                   " bytes needed, above the static " + std::to_string((size_t)SG_NOALLOC_SCRATCH_BYTES));
  int dev = 0;
  SG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return sg_fail(SG_ERR_INVALID, "pcg_solve_noalloc: device index out of range");
  if (dev != op->device)
    return sg_fail(SG_ERR_INVALID, "pcg_solve_noalloc: the operator was created on device " +
                                   std::to_string(op->device) + ", the current device is " + std::to_string(dev));
  void* ptr = nullptr;
  {
    // set-up, once per device with that device current: the host-side name of
    // the array is not a device address, so look the address up.
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_pcg_scratch);
      if (e != cudaSuccess || !p)
        return sg_fail(SG_ERR_CUDA, std::string("pcg_solve_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    ptr = g_scratch_addr[dev];
  }
  // The PCG state (reduction counters included) is reset on the stream by
  // k_pcg_setup, and the cached 1/diag(A) is revalidated by its device tag, so
  // the array's leftover contents from an earlier call are harmless.
  unsigned char* ws = static_cast<unsigned char*>(ptr);
  cudaStream_t s = as_stream(stream);
  if (op->dtype == SG_F64)
    return pcg_run<double, true>(op, static_cast<const double*>(b), static_cast<double*>(x), tol, maxit,
                                 criterion, ws, L, iters, relres, s);
  return pcg_run<float, true>(op, static_cast<const float*>(b), static_cast<float*>(x), tol, maxit,
                              criterion, ws, L, iters, relres, s);
}

// ---------------------------------------------------------------- mixed precision
// FP32 operator/PCG inside FP64 iterative refinement.  Outer loop (FP64):
// r = b - A64 x (the true-residual pass of the FP64 operator); stop when
// ||r|| <= tol ||b||; inner FP32 Jacobi-PCG solves A32 d = r to inner_tol
// (relative), x += d in FP64.  FP64 arithmetic on the GPU is confined to the
// outer residual, its norms and the correction.

template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ src, D* __restrict__ dst, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

__global__ void k_add_correction(double* __restrict__ x, const float* __restrict__ d, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

namespace {
struct IrLayout { size_t state, partials, r64, r32, d32, ws32, total; PcgLayout L32; };

IrLayout ir_layout(sg_op_t op64, sg_op_t op32) {
  IrLayout I{};
  const size_t n = (size_t)op64->n;
  const PcgLayout L64 = layout_for(op64);
  I.L32 = layout_for(op32);
  size_t off = 0;
  I.state = off; off += align_up(sizeof(PcgState));
  I.partials = off; off += align_up(sizeof(double) * 4 * (size_t)L64.max_blocks);
  I.r64 = off; off += align_up(8 * n);
  I.r32 = off; off += align_up(4 * n);
  I.d32 = off; off += align_up(4 * n);
  I.ws32 = off; off += I.L32.total;
  I.total = off;
  return I;
}

int flat_blocks(int64_t n) {
  int64_t b = (n + 255) / 256, cap = 16LL * sg_num_sms();
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

bool same_geometry(sg_op_t a, sg_op_t b) {
  return a->n == b->n && a->g.p == b->g.p && a->g.ex == b->g.ex && a->g.ey == b->g.ey &&
         a->g.ez == b->g.ez && a->lambda == b->lambda;
}
}  // namespace

extern "C" int sg_convert(const void* src, int src_dtype, void* dst, int dst_dtype, int64_t n, void* stream) {
  if (!src || !dst || n < 0 || n >= (1LL << 31)) return sg_fail(SG_ERR_INVALID, "convert: bad argument");
  cudaStream_t s = as_stream(stream);
  const int nb = flat_blocks(n);
  if (src_dtype == SG_F64 && dst_dtype == SG_F32)
    k_convert<double, float><<<nb, 256, 0, s>>>(static_cast<const double*>(src), static_cast<float*>(dst), (int)n);
  else if (src_dtype == SG_F32 && dst_dtype == SG_F64)
    k_convert<float, double><<<nb, 256, 0, s>>>(static_cast<const float*>(src), static_cast<double*>(dst), (int)n);
  else
    return sg_fail(SG_ERR_INVALID, "convert: only F64 <-> F32");
  SG_LAUNCH_CHECK("k_convert");
  return SG_OK;
}

extern "C" size_t sg_ir_workspace_bytes(sg_op_t op64, sg_op_t op32) {
  if (!op64 || !op32) return 0;
  return ir_layout(op64, op32).total;
}

// Relative tolerance of one inner solve.  A correction that reduces the
// current residual (relative size rel) by tol / rel already meets the outer
// target, so the last outer step is not solved tighter than that (with a
// factor 2 of margin); inner_tol is the floor and 0.1 the ceiling.
double ir_inner_tol(double inner_tol, double tol, double rel) { return ir_seg_tol(inner_tol, tol, rel); }

extern "C" int sg_ir_solve(sg_op_t op64, sg_op_t op32, const void* b, void* x, double tol, double inner_tol,
                           int max_outer, int maxit_inner, void* workspace, int* outer_iters,
                           int* inner_iters, double* relres, void* stream) {
  if (!op64 || !op32 || !b || !x || !workspace) return sg_fail(SG_ERR_INVALID, "ir_solve: NULL argument");
  if (op64->dtype != SG_F64 || op32->dtype != SG_F32)
    return sg_fail(SG_ERR_INVALID, "ir_solve: needs an FP64 and an FP32 operator");
  if (!same_geometry(op64, op32)) return sg_fail(SG_ERR_INVALID, "ir_solve: operators differ in mesh or lambda");
  if (!(tol > 0.0) || !(inner_tol > 0.0)) return sg_fail(SG_ERR_INVALID, "ir_solve: tolerances must be > 0");
  if (max_outer < 0 || maxit_inner < 0) return sg_fail(SG_ERR_INVALID, "ir_solve: iteration limits must be >= 0");
  if (!aligned16(b) || !aligned16(x)) return sg_fail(SG_ERR_INVALID, "ir_solve: vectors must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return sg_fail(SG_ERR_INVALID, "ir_solve: workspace must be 256-byte aligned");
  const IrLayout I = ir_layout(op64, op32);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  PcgState* st = reinterpret_cast<PcgState*>(ws + I.state);
  double* partials = reinterpret_cast<double*>(ws + I.partials);
  double* r64 = reinterpret_cast<double*>(ws + I.r64);
  float* r32 = reinterpret_cast<float*>(ws + I.r32);
  float* d32 = reinterpret_cast<float*>(ws + I.d32);
  const double* b64 = static_cast<const double*>(b);
  double* x64 = static_cast<double*>(x);
  const int n = (int)op64->n;
  const int nb = flat_blocks(n);
  cudaStream_t s = as_stream(stream);
  k_mask_faces<double><<<64, 256, 0, s>>>(x64, op64->g.nx, op64->g.ny, op64->g.nz);
  SG_LAUNCH_CHECK("k_mask_faces");
  int outer = 0, inner_total = 0;
  double rel = 0.0;
  PcgState hs;
  while (true) {
    k_pcg_setup<<<1, 32, 0, s>>>(st, tol, 0, SG_STOP_REL_B, nullptr);
    SG_LAUNCH_CHECK("k_pcg_setup");
    SemArgs<double> a{};
    a.x = x64; a.aux = b64; a.out = r64; a.partials = partials; a.st = st; a.final_pass = 1;
    int rc = sg_sem_launch<double, 2>(op64->g, a, s, 0);
    if (rc) return rc;
    SG_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaStreamSynchronize(s));
    rel = hs.bb > 0 ? sqrt(hs.rr_true / hs.bb) : sqrt(hs.rr_true);
    if (!std::isfinite(rel)) return sg_fail(SG_ERR_BREAKDOWN, "ir_solve: non-finite residual");
    if (rel <= tol || outer >= max_outer) break;
    k_convert<double, float><<<nb, 256, 0, s>>>(r64, r32, n);
    SG_LAUNCH_CHECK("k_convert");
    SG_CUDA_TRY(cudaMemsetAsync(d32, 0, sizeof(float) * (size_t)n, s));
    int it = 0;
    rc = pcg_run<float>(op32, r32, d32, ir_inner_tol(inner_tol, tol, rel), maxit_inner, SG_STOP_REL_B, ws + I.ws32,
                        I.L32, &it, nullptr, s);
    if (rc < 0) return rc;
    inner_total += it;
    k_add_correction<<<nb, 256, 0, s>>>(x64, d32, n);
    SG_LAUNCH_CHECK("k_add_correction");
    ++outer;
  }
  if (outer_iters) *outer_iters = outer;
  if (inner_iters) *inner_iters = inner_total;
  if (relres) *relres = rel;
  if (rel > tol) {
    sg_set_error("ir_solve: maximum outer iteration count reached");
    return SG_NOT_CONVERGED;
  }
  return SG_OK;
}

// ---------------------------------------------------------------- FP32 PCG with FP64 residual replacement
// Restarted refinement (sg_ir_solve) begins every inner solve from d = 0 and
// loses its Krylov space; FP32 CG then needs about twice the FP64 iteration
// count.  Here one FP32 PCG runs across the whole solve and its residual is
// replaced by the FP64 one at "reliable updates" (residual replacement: van der
// Vorst & Ye, SIAM J. Sci. Comput. 22 (2000); the mixed-precision form of
// Clark et al., Comput. Phys. Commun. 181 (2010)): whenever the FP32
// recursive residual has dropped by delta since the last update,
//   x64 += x32, x32 = 0;  r64 = b - A64 x64;  r32 = (float) r64;
//   z = r32 / diag(A);  beta = (r32.z) / (r.z)_previous;  p, q kept,
// so the next operator step forms p = z + beta p, q = A z + beta q and CG
// continues with its search direction.  The solution is accumulated and the
// stopping test taken in FP64.

// Start of a segment after an FP64 update: r32 = (float) r64, z = r32 / diag,
// r.r and r.z; the last block continues the PCG state (first = 0) with the
// new residual and sets the segment's threshold (seg_tol relative to it).
// When the true residual is more than twice the FP32 recursive one it ended
// the segment with, the two have drifted apart and the kept direction no
// longer fits: the search direction restarts (first = 1, p = z).
__global__ void __launch_bounds__(256) k_ru_restart(const double* __restrict__ r64, float* __restrict__ r32,
                                                   const float* __restrict__ invd, float* __restrict__ z, int n,
                                                   double seg_tol, PcgState* st, double* partials) {
  __shared__ double sred[64];
  double rr = 0.0, rz = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float rv = (float)r64[i];
    const float zv = rv * invd[i];
    r32[i] = rv;
    z[i] = zv;
    rr += (double)rv * rv;
    rz += (double)rv * zv;
  }
  double v[2] = {rr, rz}, tot[2];
  if (grid_reduce_last<2>(v, partials, &st->counter[1], sred, tot)) {
    if (threadIdx.x == 0) {
      const double rz_old = st->rz;
      const double rr_rec = st->rr;
      st->rr = tot[0];
      st->thr2 = seg_tol * seg_tol * tot[0];
      st->first = (tot[0] > 4.0 * rr_rec) ? 1 : 0;
      st->done = 0;
      st->status = PCG_RUNNING;
      if (!isfinite(tot[0]) || !isfinite(tot[1]) || !(rz_old > 0.0)) { st->status = PCG_BREAKDOWN; st->done = 1; }
      else {
        st->beta = st->first ? 0.0 : tot[1] / rz_old;
        st->rz = tot[1];
        if (st->iter >= st->maxit) { st->status = PCG_MAXIT; st->done = 1; }
      }
    }
  }
}

__global__ void k_add_correction_reset(double* __restrict__ x, float* __restrict__ d, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] += (double)d[i];
    d[i] = 0.f;
  }
}

extern "C" int sg_ir_solve_ru(sg_op_t op64, sg_op_t op32, const void* b, void* x, double tol, double delta,
                              int max_updates, int maxit_inner, void* workspace, int* updates, int* inner_iters,
                              double* relres, void* stream) {
  if (!op64 || !op32 || !b || !x || !workspace) return sg_fail(SG_ERR_INVALID, "ir_solve_ru: NULL argument");
  if (op64->dtype != SG_F64 || op32->dtype != SG_F32)
    return sg_fail(SG_ERR_INVALID, "ir_solve_ru: needs an FP64 and an FP32 operator");
  if (!same_geometry(op64, op32)) return sg_fail(SG_ERR_INVALID, "ir_solve_ru: operators differ in mesh or lambda");
  if (!(tol > 0.0) || !(delta > 0.0) || !(delta < 1.0)) return sg_fail(SG_ERR_INVALID, "ir_solve_ru: need tol > 0, 0 < delta < 1");
  if (max_updates < 0 || maxit_inner < 0) return sg_fail(SG_ERR_INVALID, "ir_solve_ru: iteration limits must be >= 0");
  if (!aligned16(b) || !aligned16(x)) return sg_fail(SG_ERR_INVALID, "ir_solve_ru: vectors must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return sg_fail(SG_ERR_INVALID, "ir_solve_ru: workspace must be 256-byte aligned");
  const IrLayout I = ir_layout(op64, op32);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  unsigned char* ws32 = ws + I.ws32;
  PcgState* st64 = reinterpret_cast<PcgState*>(ws + I.state);
  PcgState* st32 = reinterpret_cast<PcgState*>(ws32 + I.L32.state);
  double* partials = reinterpret_cast<double*>(ws + I.partials);
  double* r64 = reinterpret_cast<double*>(ws + I.r64);
  float* r32 = reinterpret_cast<float*>(ws + I.r32);
  float* d32 = reinterpret_cast<float*>(ws + I.d32);
  const double* b64 = static_cast<const double*>(b);
  double* x64 = static_cast<double*>(x);
  const int n = (int)op64->n;
  const int nb = flat_blocks(n);
  cudaStream_t s = as_stream(stream);
  auto fp64_residual = [&]() -> int {     // r64 = b - A64 x64, ||r64||^2 and ||b||^2 into st64
    k_pcg_setup<<<1, 32, 0, s>>>(st64, tol, 0, SG_STOP_REL_B, nullptr);
    SG_LAUNCH_CHECK("k_pcg_setup");
    SemArgs<double> a{};
    a.x = x64; a.aux = b64; a.out = r64; a.partials = partials; a.st = st64; a.final_pass = 1;
    return sg_sem_launch<double, 2>(op64->g, a, s, 0);
  };
  k_mask_faces<double><<<64, 256, 0, s>>>(x64, op64->g.nx, op64->g.ny, op64->g.nz);
  SG_LAUNCH_CHECK("k_mask_faces");
  int rc = fp64_residual();
  if (rc) return rc;
  PcgState h64, h32;
  int nupd = 0, inner = 0;
  cudaGraphExec_t exec = nullptr;
  // one segment after its start: the FP32 iterations, x64 += x32, the FP64
  // residual, and the host reads both states (the segment's one synchronisation)
  auto run_segment = [&]() -> int {
    if (!exec && !sg_profiling_on()) exec = iteration_graph<float>(op32, ws32, I.L32);
    if (exec) {
      SG_CUDA_TRY(cudaGraphLaunch(exec, s));
    } else {
      const int r2 = pcg_iterate_launches<float, false>(op32, d32, maxit_inner, ws32, I.L32, s);
      if (r2) return r2;
    }
    k_add_correction_reset<<<nb, 256, 0, s>>>(x64, d32, n);
    SG_LAUNCH_CHECK("k_add_correction_reset");
    const int r3 = fp64_residual();
    if (r3) return r3;
    SG_CUDA_TRY(cudaMemcpyAsync(&h32, st32, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaMemcpyAsync(&h64, st64, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaStreamSynchronize(s));
    return SG_OK;
  };
  double bb = 0.0, rel = 0.0;
  bool more = true;
  if (max_updates > 0) {
    // first segment: PCG from x32 = 0 on r32 = (float) r64, enqueued before
    // the host has seen the initial residual -- k_ru_first_tol takes the
    // segment's tolerance from it on the device, or turns the segment into a
    // no-op when the residual already meets tol (one synchronisation less per
    // call: the 16^3 p = 7 FP32 + replacement step 0.783 -> 0.768 ms)
    k_convert<double, float><<<nb, 256, 0, s>>>(r64, r32, n);
    SG_LAUNCH_CHECK("k_convert");
    SG_CUDA_TRY(cudaMemsetAsync(d32, 0, sizeof(float) * (size_t)n, s));
    rc = pcg_start<float>(op32, r32, d32, delta, maxit_inner, SG_STOP_REL_B, ws32, I.L32, s, st64, delta, tol);
    if (rc) return rc;
    rc = run_segment();
    if (rc) return rc;
    bb = h64.bb;
    rel = bb > 0 ? sqrt(h64.rr_true / bb) : sqrt(h64.rr_true);
    if (!std::isfinite(rel)) return sg_fail(SG_ERR_BREAKDOWN, "ir_solve_ru: non-finite residual");
    if (!h32.pad[0]) {              // the segment ran (pad[0]: skipped by k_ru_first_tol)
      if (exec) sg_count_launches(2 * (h32.iter > 0 ? h32.iter : 1));
      ++nupd;
      inner = h32.iter;
      if (h32.status == PCG_BREAKDOWN) return sg_fail(SG_ERR_BREAKDOWN, "ir_solve_ru: breakdown");
      if (h32.status == PCG_MAXIT) more = false;
    }
  } else {
    SG_CUDA_TRY(cudaMemcpyAsync(&h64, st64, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaStreamSynchronize(s));
    bb = h64.bb;
    rel = bb > 0 ? sqrt(h64.rr_true / bb) : sqrt(h64.rr_true);
    if (!std::isfinite(rel)) return sg_fail(SG_ERR_BREAKDOWN, "ir_solve_ru: non-finite residual");
  }
  while (more && rel > tol && nupd < max_updates) {
    // later segments: residual replaced, search direction kept
    const double seg_tol = ir_inner_tol(delta, tol, rel);
    k_ru_restart<<<update_blocks(op32->n, 4), 256, 0, s>>>(r64, reinterpret_cast<float*>(ws32 + I.L32.r),
                                                          reinterpret_cast<const float*>(ws32 + I.L32.invd),
                                                          reinterpret_cast<float*>(ws32 + I.L32.z), n, seg_tol, st32,
                                                          reinterpret_cast<double*>(ws32 + I.L32.partials));
    SG_LAUNCH_CHECK("k_ru_restart");
    rc = run_segment();
    if (rc) return rc;
    ++nupd;
    if (exec) sg_count_launches(2 * (h32.iter - inner > 0 ? h32.iter - inner : 1));
    inner = h32.iter;
    rel = bb > 0 ? sqrt(h64.rr_true / bb) : sqrt(h64.rr_true);
    if (!std::isfinite(rel) || h32.status == PCG_BREAKDOWN) return sg_fail(SG_ERR_BREAKDOWN, "ir_solve_ru: breakdown");
    if (h32.status == PCG_MAXIT) break;
  }
  if (updates) *updates = nupd;
  if (inner_iters) *inner_iters = inner;
  if (relres) *relres = rel;
  if (rel > tol) {
    sg_set_error("ir_solve_ru: update or inner iteration limit reached");
    return SG_NOT_CONVERGED;
  }
  return SG_OK;
}
