// sg_batch.cu -- several independent solve sequences advanced together.
//
// The paper keeps separate history spaces for the three velocity components
// and the pressure (Sec. 6.1, GPU implementation) and solves each system with
// PCG (Sec. 5.3).  Here up to SG_BATCH_MAX such systems, each on its own mesh
// (same degree p, any size and lambda), run their FP32 Jacobi-PCG iterations
// in ONE persistent cooperative launch per CG iteration:
//   phase A  operator work items of every unconverged system (w = A z; p, q
//            updated in place; p.q per system), then a grid barrier;
//   alpha    every CTA sums the per-CTA p.q partials in CTA order;
//   phase B  x += alpha p, r -= alpha q, z = r / diag(A), r.r, r.z per system,
//            then a grid barrier; CTA 0 finalises beta, the iteration count
//            and the convergence flag of every system.
// The launches are replayed from a CUDA graph (a fixed number per replay;
// iterations after convergence return at once); the host reads the done
// flags once per replay.  FP64 iterative refinement wraps the inner solve:
// the outer FP64 residual of each system uses its FP64 operator.
// Grid barriers spin with an iteration limit; on expiry they set an error
// flag (reported as SG_ERR_TIMEOUT) instead of waiting forever.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sg_sem_launch.cuh"

namespace {
constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr int BP = 7;                       // degree of the batched kernel
using BTile = SemTile<BP>;
constexpr long long kSpinLimit = 1LL << 24; // grid-barrier polls before giving up
}

struct BatchSeq {
  SemGeom g;
  float *x, *r, *z, *p, *q;
  const float* invd;
  const float* b;
  int n, zl;
  PcgState* st;
};

struct BatchArgs {
  BatchSeq seq[SG_BATCH_MAX];
  int nseq;
  const int4* items;        // (system, tile x, tile y, first layer)
  int nitems;
  double* partials;         // [block][3 * SG_BATCH_MAX]
  unsigned int* bar;        // [0] arrivals, [1] generation
  int* err;
  int nblocks;
  cudaGraphConditionalHandle cond;   // WHILE condition of the iteration graph (use_cond)
  int use_cond;
  int solo_tail;            // use_cond: end the loop when one system is left running
};

// Grid-wide barrier for a cooperative launch, bounded spin (error flag on expiry).
__device__ __forceinline__ void grid_barrier(unsigned int* bar, int* err, unsigned int nblocks,
                                             long long spin_limit = kSpinLimit) {
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile unsigned int* gen = bar + 1;
    const unsigned int g0 = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g0) {
        if (++it > spin_limit) { atomicExch(err, 1); break; }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ void block_sum_2d(double (&v)[NV], double* smem) { block_sum<NV>(v, smem); }

// COND: the launch is the body of a conditional WHILE node and sets its
// condition; the other instantiation (replay graphs) contains no conditional
// call, which keeps its graph nodes visible to kernel profilers.
template <bool COND>
__global__ void __launch_bounds__(BTile::NTHREADS, 3) k_batch_iter(const __grid_constant__ BatchArgs A) {
  constexpr int NS = SG_BATCH_MAX;
  __shared__ float s_beta[NS];
  __shared__ int s_first[NS], s_done[NS];
  __shared__ float s_alpha[NS];
  __shared__ double sred[32 * 2 * NS];
  __shared__ int s_all_done;
  __shared__ SemTabs<float, BP> s_tabs;
  const int tid = threadIdx.x + BTile::TX * threadIdx.y;
  const int NT = BTile::NTHREADS;
  if (tid == 0) {
    int all = 1;
    for (int s = 0; s < NS; ++s) {
      if (s < A.nseq) {
        s_done[s] = A.seq[s].st->done;
        s_beta[s] = (float)A.seq[s].st->beta;
        s_first[s] = A.seq[s].st->first;
      } else {
        s_done[s] = 1; s_beta[s] = 0.f; s_first[s] = 1;
      }
      all &= s_done[s];
    }
    // an expired barrier wait in an earlier launch stops the iterations (the
    // flag was written before this launch began, so every CTA reads the same)
    s_all_done = all || *(volatile int*)A.err;
  }
  __syncthreads();
  if (s_all_done) {         // uniform over the grid: no barrier is entered
    if constexpr (COND) {
      if (A.use_cond && blockIdx.x == 0 && tid == 0) cudaGraphSetConditional(A.cond, 0u);
    }
    return;
  }

  // ---- phase A: operator items
  float pq[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) pq[s] = 0.f;
  for (int it = blockIdx.x; it < A.nitems; it += gridDim.x) {
    const int4 w = A.items[it];
    if (s_done[w.x]) continue;
    const BatchSeq& S = A.seq[w.x];
    SemArgs<float> a{};
    a.x = S.z; a.out = S.q; a.out2 = S.p;
    float red[3] = {0.f, 0.f, 0.f};
    const int e1 = min(S.g.ez, w.w + S.zl);
    // this system's coefficients into shared memory (after the previous item
    // is done with the last copy)
    __syncthreads();
    {
      constexpr int NW = (int)(sizeof(SemTabs<float, BP>) / sizeof(float));
      const float* src = static_cast<const float*>(S.g.tabs);
      float* dst = reinterpret_cast<float*>(&s_tabs);
      for (int i = tid; i < NW; i += NT) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    sem_item<float, BP, 1, true>(S.g, s_tabs, a, w.y, w.z, w.w, e1, &s_beta[w.x], &s_first[w.x], red, nullptr,
                                 false);
#pragma unroll
    for (int s = 0; s < NS; ++s)
      if (s == w.x) pq[s] += red[0];
  }
  {
    double v[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) v[s] = (double)pq[s];
    block_sum<NS>(v, sred);
    if (tid == 0)
      for (int s = 0; s < NS; ++s) A.partials[(size_t)blockIdx.x * 3 * NS + s] = v[s];
  }
  grid_barrier(A.bar, A.err, A.nblocks);

  // ---- alpha per system: every CTA sums the partials in CTA order
  {
    double v[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) v[s] = 0.0;
    for (int b = tid; b < A.nblocks; b += NT)
#pragma unroll
      for (int s = 0; s < NS; ++s) v[s] += __ldcg(&A.partials[(size_t)b * 3 * NS + s]);
    block_sum<NS>(v, sred);
    if (tid == 0)
      for (int s = 0; s < NS; ++s) {
        const double rz = (s < A.nseq) ? A.seq[s].st->rz : 0.0;
        s_alpha[s] = (v[s] > 0.0) ? (float)(rz / v[s]) : 0.f;
        if (blockIdx.x == 0 && s < A.nseq && !s_done[s]) {
          A.seq[s].st->pq = v[s];
          if (!(v[s] > 0.0) || !isfinite(v[s])) { A.seq[s].st->status = PCG_BREAKDOWN; }
        }
      }
    __syncthreads();
  }

  // ---- phase B: vector updates of every unconverged system
  float rr[NS], rzv[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) { rr[s] = 0.f; rzv[s] = 0.f; }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    if (s >= A.nseq || s_done[s]) continue;
    const BatchSeq& S = A.seq[s];
    const float al = s_alpha[s];
    const int nv = S.n / 4;
    for (int i = blockIdx.x * NT + tid; i < nv; i += gridDim.x * NT) {
      float4 xv = reinterpret_cast<float4*>(S.x)[i];
      const float4 pv = reinterpret_cast<const float4*>(S.p)[i];
      float4 rv = reinterpret_cast<float4*>(S.r)[i];
      const float4 qv = reinterpret_cast<const float4*>(S.q)[i];
      const float4 dv = reinterpret_cast<const float4*>(S.invd)[i];
      float4 zv;
      xv.x += al * pv.x; rv.x -= al * qv.x; zv.x = rv.x * dv.x;
      xv.y += al * pv.y; rv.y -= al * qv.y; zv.y = rv.y * dv.y;
      xv.z += al * pv.z; rv.z -= al * qv.z; zv.z = rv.z * dv.z;
      xv.w += al * pv.w; rv.w -= al * qv.w; zv.w = rv.w * dv.w;
      rr[s] += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
      rzv[s] += rv.x * zv.x + rv.y * zv.y + rv.z * zv.z + rv.w * zv.w;
      reinterpret_cast<float4*>(S.x)[i] = xv;
      reinterpret_cast<float4*>(S.r)[i] = rv;
      reinterpret_cast<float4*>(S.z)[i] = zv;
    }
    for (int i = nv * 4 + blockIdx.x * NT + tid; i < S.n; i += gridDim.x * NT) {
      S.x[i] += al * S.p[i];
      const float rs = S.r[i] - al * S.q[i];
      const float zs = rs * S.invd[i];
      S.r[i] = rs; S.z[i] = zs;
      rr[s] += rs * rs; rzv[s] += rs * zs;
    }
  }
  {
    double v[2 * NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) { v[s] = (double)rr[s]; v[NS + s] = (double)rzv[s]; }
    block_sum<2 * NS>(v, sred);
    if (tid == 0)
      for (int k = 0; k < 2 * NS; ++k) A.partials[(size_t)blockIdx.x * 3 * NS + NS + k] = v[k];
  }
  grid_barrier(A.bar, A.err, A.nblocks);

  // ---- CTA 0 finalises every system
  if (blockIdx.x == 0) {
    double v[2 * NS];
#pragma unroll
    for (int k = 0; k < 2 * NS; ++k) v[k] = 0.0;
    for (int b = tid; b < A.nblocks; b += NT)
#pragma unroll
      for (int k = 0; k < 2 * NS; ++k) v[k] += __ldcg(&A.partials[(size_t)b * 3 * NS + NS + k]);
    block_sum<2 * NS>(v, sred);
    if (tid == 0) {
      for (int s = 0; s < A.nseq; ++s) {
        if (s_done[s]) continue;
        PcgState* st = A.seq[s].st;
        st->iter += 1;
        st->first = 0;
        st->alpha = s_alpha[s];
        const double rrs = v[s], rzs = v[NS + s];
        st->rr = rrs;
        if (st->status == PCG_BREAKDOWN || !isfinite(rrs) || !isfinite(rzs)) { st->status = PCG_BREAKDOWN; st->done = 1; }
        else if (rrs <= st->thr2) { st->status = PCG_CONVERGED; st->done = 1; }
        else {
          st->beta = rzs / st->rz;
          st->rz = rzs;
          if (st->iter >= st->maxit) { st->status = PCG_MAXIT; st->done = 1; }
        }
      }
      if constexpr (COND) {
        if (A.use_cond) {     // continue while systems run and no barrier wait expired
          int running = 0;
          for (int s = 0; s < A.nseq; ++s) running += !A.seq[s].st->done;
          // with solo_tail the last running system continues in its own
          // (non-persistent) iteration graph, launched by the host
          int more = running > (A.solo_tail ? 1 : 0);
          if (*(volatile int*)A.err) more = 0;
          cudaGraphSetConditional(A.cond, more ? 1u : 0u);
        }
      }
    }
  }
}

// Start of a batched inner solve from x = 0: r = b, z = r / diag(A),
// r.r, r.z, b.b per system; blockIdx.y selects the system.
struct BatchTol { double rel[SG_BATCH_MAX]; };

__global__ void __launch_bounds__(256) k_batch_init(const __grid_constant__ BatchArgs A, BatchTol tol, int maxit, unsigned int* counters,
                                                    const int* active) {
  __shared__ double sred[32 * 3];
  const int s = blockIdx.y;
  if (s >= A.nseq) return;
  const BatchSeq& S = A.seq[s];
  if (!active[s]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) { S.st->done = 1; S.st->status = PCG_CONVERGED; S.st->iter = 0; }
    return;
  }
  float rr = 0.f, rz = 0.f, bb = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.n; i += gridDim.x * blockDim.x) {
    const float bv = S.b[i];
    const float zv = bv * S.invd[i];
    S.x[i] = 0.f;
    S.r[i] = bv;
    S.z[i] = zv;
    rr += bv * bv; rz += bv * zv; bb += bv * bv;
  }
  double v[3] = {(double)rr, (double)rz, (double)bb};
  block_sum<3>(v, sred);
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    double* part = A.partials + ((size_t)s * gridDim.x + blockIdx.x) * 3;
    part[0] = v[0]; part[1] = v[1]; part[2] = v[2];
    __threadfence();
    s_last = (atomicAdd(&counters[s], 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double acc[3] = {0.0, 0.0, 0.0};
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const double* part = A.partials + ((size_t)s * gridDim.x + b) * 3;
    acc[0] += __ldcg(part); acc[1] += __ldcg(part + 1); acc[2] += __ldcg(part + 2);
  }
  block_sum<3>(acc, sred);
  if (threadIdx.x == 0) {
    counters[s] = 0u;
    PcgState* st = S.st;
    st->rr = acc[0]; st->rz = acc[1]; st->bb = acc[2]; st->rr0 = acc[0];
    st->thr2 = tol.rel[s] * tol.rel[s] * acc[2];
    st->iter = 0; st->first = 1; st->beta = 0.0; st->maxit = maxit;
    st->status = PCG_RUNNING; st->done = 0;
    if (!isfinite(acc[0])) { st->status = PCG_BREAKDOWN; st->done = 1; }
    else if (acc[0] <= st->thr2) { st->status = PCG_CONVERGED; st->done = 1; }
    else if (maxit <= 0) { st->status = PCG_MAXIT; st->done = 1; }
  }
}

__global__ void k_pcg_state_reset_counters(PcgState* st) {
  if (threadIdx.x < 4 && blockIdx.x == 0) st->counter[threadIdx.x] = 0u;
}

__global__ void k_convert_fill(float* v, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = 1.0f;
}

__global__ void k_batch_add(double* x, const float* d, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] += (double)d[i];
}

__global__ void k_batch_to_f32(const double* r, float* b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (float)r[i];
}

template <typename T>
__global__ void k_batch_mask(T* v, int nx, int ny, int nz) {
  const size_t nxy = (size_t)nx * ny;
  const int stride = gridDim.x * blockDim.x, t0 = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = t0; i < nx * ny; i += stride) { v[i] = (T)0; v[(size_t)(nz - 1) * nxy + i] = (T)0; }
  for (int i = t0; i < nx * nz; i += stride) {
    int xi = i % nx, zi = i / nx;
    v[(size_t)zi * nxy + xi] = (T)0; v[(size_t)zi * nxy + (size_t)(ny - 1) * nx + xi] = (T)0;
  }
  for (int i = t0; i < ny * nz; i += stride) {
    int yi = i % ny, zi = i / ny;
    v[(size_t)zi * nxy + (size_t)yi * nx] = (T)0; v[(size_t)zi * nxy + (size_t)yi * nx + nx - 1] = (T)0;
  }
}

__global__ void k_batch_invdiag(const SemGeom g, FastDiv dnx, FastDiv dnxy, int n, float* out) {
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
    out[i] = (float)(1.0 / v);
  }
}

// ---------------------------------------------------------------- host side
struct sg_batch_s {
  int nseq;
  sg_op_t op64[SG_BATCH_MAX], op32[SG_BATCH_MAX];
  unsigned char* ws;
  size_t off_state, off_partials, off_bar, off_items, off_counters, off_active, off_ir;
  size_t off_vec[SG_BATCH_MAX][7];   // x, r, z, p, q, invd, b (FP32) ; r64 in off_ir
  size_t off_r64[SG_BATCH_MAX];
  int max_items, max_blocks;
  // tuned launch configuration
  int zl, blocks_per_sm, nitems, nblocks, tuned;
  int graph_iters;
  cudaGraphExec_t solo[SG_BATCH_MAX];   // per-system iteration graphs (single-system tail)
  cudaGraphExec_t graph;
  int graph_ready;
  int graph_while;          // 1: the graph is one WHILE node (one launch per solve)
  int graph_prof;           // the graph was built while kernel timing was on (replay form)
  cudaStream_t graph_stream;
};

namespace {

int n_tiles(const SemGeom& g, int zl) {
  return ((g.ex + BTile::TEX - 1) / BTile::TEX) * ((g.ey + BTile::TEY - 1) / BTile::TEY) * ((g.ez + zl - 1) / zl);
}

size_t batch_smem() {
  return sizeof(float) * ((size_t)BTile::NPL * BTile::PY * BTile::template pitch<float>() +
                          2 * (size_t)BP * BTile::TY * BTile::TX);
}

struct BLayout {
  size_t state, partials, bar, items, counters, active, vec[SG_BATCH_MAX][7], r64[SG_BATCH_MAX], total;
  int max_items, max_blocks;
};

BLayout blayout(int nseq, const sg_op_t* ops) {
  BLayout L{};
  int items = 0;
  for (int s = 0; s < nseq; ++s) items += n_tiles(ops[s]->g, 1);
  L.max_items = items;
  L.max_blocks = 16 * sg_num_sms();
  size_t off = 0;
  L.state = off; off += align_up(sizeof(PcgState) * SG_BATCH_MAX);
  // per-block partials of the persistent kernel and of the FP64 residual
  // launches, whose CTA count is at most the one-layer tile count (items)
  size_t pb = (size_t)(L.max_blocks > 4096 ? L.max_blocks : 4096);
  if ((size_t)items > pb) pb = (size_t)items;
  L.partials = off; off += align_up(sizeof(double) * 3 * SG_BATCH_MAX * pb);
  L.bar = off; off += align_up(sizeof(unsigned int) * 4 + sizeof(int) * 4);
  L.items = off; off += align_up(sizeof(int4) * (size_t)items);
  L.counters = off; off += align_up(sizeof(unsigned int) * SG_BATCH_MAX);
  L.active = off; off += align_up(sizeof(int) * SG_BATCH_MAX);
  for (int s = 0; s < nseq; ++s) {
    const size_t vb = align_up(4 * (size_t)ops[s]->n);
    for (int k = 0; k < 7; ++k) { L.vec[s][k] = off; off += vb; }
    L.r64[s] = off; off += align_up(8 * (size_t)ops[s]->n);
  }
  L.total = off;
  return L;
}

BatchArgs make_args(sg_batch_t b) {
  BatchArgs A{};
  A.nseq = b->nseq;
  for (int s = 0; s < b->nseq; ++s) {
    BatchSeq& S = A.seq[s];
    S.g = b->op32[s]->g;
    S.x = reinterpret_cast<float*>(b->ws + b->off_vec[s][0]);
    S.r = reinterpret_cast<float*>(b->ws + b->off_vec[s][1]);
    S.z = reinterpret_cast<float*>(b->ws + b->off_vec[s][2]);
    S.p = reinterpret_cast<float*>(b->ws + b->off_vec[s][3]);
    S.q = reinterpret_cast<float*>(b->ws + b->off_vec[s][4]);
    S.invd = reinterpret_cast<const float*>(b->ws + b->off_vec[s][5]);
    S.b = reinterpret_cast<const float*>(b->ws + b->off_vec[s][6]);
    S.n = (int)b->op32[s]->n;
    S.zl = b->zl;
    S.st = reinterpret_cast<PcgState*>(b->ws + b->off_state) + s;
  }
  A.items = reinterpret_cast<const int4*>(b->ws + b->off_items);
  A.nitems = b->nitems;
  A.partials = reinterpret_cast<double*>(b->ws + b->off_partials);
  A.bar = reinterpret_cast<unsigned int*>(b->ws + b->off_bar);
  A.err = reinterpret_cast<int*>(b->ws + b->off_bar + 4 * sizeof(unsigned int));
  A.nblocks = b->nblocks;
  return A;
}

// Work items for a given z-chunk depth: larger systems first (longest work first).
int build_items(sg_batch_t b, int zl, cudaStream_t s) {
  std::vector<int4> items;
  std::vector<int> order(b->nseq);
  for (int i = 0; i < b->nseq; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int c) { return b->op32[a]->n > b->op32[c]->n; });
  for (int si : order) {
    const SemGeom& g = b->op32[si]->g;
    const int tx = (g.ex + BTile::TEX - 1) / BTile::TEX, ty = (g.ey + BTile::TEY - 1) / BTile::TEY;
    for (int e0 = 0; e0 < g.ez; e0 += zl)
      for (int by = 0; by < ty; ++by)
        for (int bx = 0; bx < tx; ++bx) items.push_back(make_int4(si, bx, by, e0));
  }
  if ((int)items.size() > b->max_items) return sg_fail(SG_ERR_INVALID, "batch: work list overflow");
  SG_CUDA_TRY(cudaMemcpyAsync(b->ws + b->off_items, items.data(), sizeof(int4) * items.size(),
                              cudaMemcpyHostToDevice, s));
  SG_CUDA_TRY(cudaStreamSynchronize(s));
  b->nitems = (int)items.size();
  b->zl = zl;
  return SG_OK;
}

int launch_iter(sg_batch_t b, cudaStream_t s, cudaGraphConditionalHandle cond = 0, int use_cond = 0) {
  BatchArgs A = make_args(b);
  A.cond = cond;
  A.use_cond = use_cond;
  A.solo_tail = use_cond && b->nseq > 1;
  void* params[] = {&A};
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(b->nblocks);
  cfg.blockDim = dim3(BTile::TX, BTile::TY);
  cfg.dynamicSmemBytes = batch_smem();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const void* fn = use_cond ? (const void*)k_batch_iter<true> : (const void*)k_batch_iter<false>;
  cudaError_t e = cudaLaunchKernelExC(&cfg, fn, params);
  sg_count_launch();
  if (e != cudaSuccess) return sg_fail(SG_ERR_CUDA, std::string("batch iteration launch: ") + cudaGetErrorString(e));
  return SG_OK;
}

int max_coresident(int* per_sm) {
  static int cached = -1;
  if (cached < 0) {
    // both instantiations: the grid must be co-resident for either
    cudaError_t e = cudaFuncSetAttribute(k_batch_iter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batch_smem());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_batch_iter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_smem());
    if (e != cudaSuccess) return sg_fail(SG_ERR_CUDA, std::string("batch smem attribute: ") + cudaGetErrorString(e));
    int nb = 0, nb2 = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_iter<true>, BTile::NTHREADS, batch_smem());
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb2, k_batch_iter<false>, BTile::NTHREADS, batch_smem());
    if (e != cudaSuccess || nb < 1 || nb2 < 1) return sg_fail(SG_ERR_CUDA, "batch occupancy query failed");
    cached = nb < nb2 ? nb : nb2;
  }
  *per_sm = cached;
  return SG_OK;
}

struct PollS { int iter, done, status, first; };

}  // namespace

extern "C" size_t sg_batch_workspace_bytes(int nseq, const sg_op_t* ops64, const sg_op_t* ops32) {
  if (nseq < 1 || nseq > SG_BATCH_MAX || !ops64 || !ops32) return 0;
  for (int s = 0; s < nseq; ++s) if (!ops32[s] || !ops64[s]) return 0;
  return blayout(nseq, ops32).total;
}

extern "C" int sg_batch_create(sg_batch_t* out, int nseq, const sg_op_t* ops64, const sg_op_t* ops32, void* workspace) {
  if (!out) return sg_fail(SG_ERR_INVALID, "batch_create: NULL output handle");
  *out = nullptr;
  if (nseq < 1 || nseq > SG_BATCH_MAX) return sg_fail(SG_ERR_INVALID, "batch_create: 1 <= nseq <= SG_BATCH_MAX");
  if (!ops64 || !ops32 || !workspace) return sg_fail(SG_ERR_INVALID, "batch_create: NULL argument");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return sg_fail(SG_ERR_INVALID, "batch_create: workspace must be 256-byte aligned");
  for (int s = 0; s < nseq; ++s) {
    if (!ops64[s] || !ops32[s]) return sg_fail(SG_ERR_INVALID, "batch_create: NULL operator");
    if (ops64[s]->dtype != SG_F64 || ops32[s]->dtype != SG_F32) return sg_fail(SG_ERR_INVALID, "batch_create: need FP64 and FP32 operators");
    if (ops32[s]->g.p != BP || ops64[s]->g.p != BP) return sg_fail(SG_ERR_INVALID, "batch_create: the batched kernel is built for p = 7");
    if (ops64[s]->n != ops32[s]->n || ops64[s]->lambda != ops32[s]->lambda) return sg_fail(SG_ERR_INVALID, "batch_create: operator pair mismatch");
  }
  BLayout L = blayout(nseq, ops32);
  sg_batch_s* b = new sg_batch_s();
  b->nseq = nseq;
  for (int s = 0; s < nseq; ++s) { b->op64[s] = ops64[s]; b->op32[s] = ops32[s]; }
  b->ws = static_cast<unsigned char*>(workspace);
  b->off_state = L.state; b->off_partials = L.partials; b->off_bar = L.bar; b->off_items = L.items;
  b->off_counters = L.counters; b->off_active = L.active;
  for (int s = 0; s < nseq; ++s) { for (int k = 0; k < 7; ++k) b->off_vec[s][k] = L.vec[s][k]; b->off_r64[s] = L.r64[s]; }
  b->max_items = L.max_items; b->max_blocks = L.max_blocks;
  b->graph_iters = 8;
  for (int k = 0; k < SG_BATCH_MAX; ++k) b->solo[k] = nullptr;
  b->graph_ready = 0;
  b->graph_while = 0;
  b->graph_prof = 0;
  int per_sm = 0;
  int rc = max_coresident(&per_sm);
  if (rc) { delete b; return rc; }
  b->blocks_per_sm = per_sm;
  b->nblocks = per_sm * sg_num_sms();
  cudaStream_t s0 = 0;
  cudaError_t e = cudaMemsetAsync(b->ws, 0, L.total, s0);
  if (e != cudaSuccess) { delete b; return sg_fail(SG_ERR_CUDA, std::string("batch_create: ") + cudaGetErrorString(e)); }
  rc = build_items(b, 2, s0);
  if (rc) { delete b; return rc; }
  for (int s = 0; s < nseq; ++s) {
    const sg_op_t op = ops32[s];
    k_batch_invdiag<<<16 * sg_num_sms(), 256, 0, s0>>>(op->g, op->div_nx, op->div_nxy, (int)op->n,
                                                      reinterpret_cast<float*>(b->ws + b->off_vec[s][5]));
    sg_count_launch();
  }
  e = cudaStreamSynchronize(s0);
  if (e != cudaSuccess) { delete b; return sg_fail(SG_ERR_CUDA, std::string("batch_create: ") + cudaGetErrorString(e)); }
  *out = b;
  return SG_OK;
}

extern "C" int sg_batch_destroy(sg_batch_t b) {
  if (b && b->graph_ready) cudaGraphExecDestroy(b->graph);
  if (b)
    for (int k = 0; k < SG_BATCH_MAX; ++k)
      if (b->solo[k]) cudaGraphExecDestroy(b->solo[k]);
  delete b;
  return SG_OK;
}

// Remaining iterations of system k alone: its state (iteration count, beta,
// r.z, direction) continues in a WHILE graph of the FP32 operator step and
// update on its own vectors (built once per system and workspace).
int sg_pcg_iteration_graph_f32(sg_op_t op, const PcgIterPtrs<float>& v, cudaGraphExec_t* out);

static int batch_solo(sg_batch_t b, int k, cudaStream_t s) {
  BatchArgs A = make_args(b);
  const BatchSeq& S = A.seq[k];
  if (!b->solo[k]) {
    PcgIterPtrs<float> v{};
    v.st = S.st; v.partials = A.partials;
    v.r = S.r; v.z = S.z; v.p = S.p; v.q = S.q; v.x = S.x; v.invd = S.invd;
    int rc = sg_pcg_iteration_graph_f32(b->op32[k], v, &b->solo[k]);
    if (rc) { b->solo[k] = nullptr; return rc; }
  }
  k_pcg_state_reset_counters<<<1, 32, 0, s>>>(S.st);
  SG_LAUNCH_CHECK("k_pcg_state_reset_counters");
  SG_CUDA_TRY(cudaGraphLaunch(b->solo[k], s));
  return SG_OK;
}

// Inner batched FP32 PCG on the systems flagged active (b: the FP32 right-hand
// sides already in the workspace).  Per-system iteration counts out.
static int batch_inner(sg_batch_t b, const int* active, const BatchTol& tol, int maxit, int* iters, cudaStream_t s) {
  BatchArgs A = make_args(b);
  SG_CUDA_TRY(cudaMemcpyAsync(b->ws + b->off_active, active, sizeof(int) * b->nseq, cudaMemcpyHostToDevice, s));
  int gx = 4 * sg_num_sms() / (b->nseq > 0 ? b->nseq : 1);
  if (gx < 1) gx = 1;
  k_batch_init<<<dim3(gx, b->nseq), 256, 0, s>>>(A, tol, maxit, reinterpret_cast<unsigned int*>(b->ws + b->off_counters),
                                                 reinterpret_cast<const int*>(b->ws + b->off_active));
  SG_LAUNCH_CHECK("k_batch_init");
  // The iterations as a CUDA graph, built once per stream: preferably a
  // conditional WHILE node around one persistent launch (CTA 0 of every
  // iteration sets the condition; one graph launch runs the whole solve),
  // else graph_iters launches replayed until every system is done.
  // With kernel timing on (sg_profile_enable) the replay form is built: its
  // kernel nodes are visible one by one to profilers, which do not look
  // inside graphs with conditional nodes.
  const int prof = sg_profiling_on() ? 1 : 0;
  if (!b->graph_ready || b->graph_stream != s || b->graph_prof != prof) {
    if (b->graph_ready) { cudaGraphExecDestroy(b->graph); b->graph_ready = 0; }
    cudaStream_t cs;
    SG_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    int rc = SG_OK;
    // WHILE form
    cudaGraphConditionalHandle cond = 0;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    cudaError_t e = prof ? cudaErrorNotSupported : cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
    }
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = launch_iter(b, cs, cond, 1);
      cudaGraph_t body = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(cs, &body);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && rc == SG_OK) e = cudaGraphInstantiate(&b->graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    b->graph_while = (e == cudaSuccess && rc == SG_OK);
    if (!b->graph_while) {
      // replay form
      cudaGetLastError();
      graph = nullptr;
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        for (int i = 0; i < b->graph_iters; ++i) {
          rc = launch_iter(b, cs);
          if (rc) { cudaStreamEndCapture(cs, &graph); if (graph) cudaGraphDestroy(graph); cudaStreamDestroy(cs); return rc; }
        }
        e = cudaStreamEndCapture(cs, &graph);
      }
      if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
      }
    }
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return sg_fail(SG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    b->graph_ready = 1;
    b->graph_stream = s;
    b->graph_prof = prof;
  }
  PollS poll[SG_BATCH_MAX];
  int done_all = 0, replays = 0;
  const int max_replays = b->graph_while ? 1 : maxit / b->graph_iters + 2;
  while (!done_all) {
    SG_CUDA_TRY(cudaGraphLaunch(b->graph, s));
    ++replays;
    for (int k = 0; k < b->nseq; ++k)
      SG_CUDA_TRY(cudaMemcpyAsync(&poll[k], &A.seq[k].st->iter, sizeof(PollS), cudaMemcpyDeviceToHost, s));
    int err = 0;
    SG_CUDA_TRY(cudaMemcpyAsync(&err, A.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SG_CUDA_TRY(cudaStreamSynchronize(s));
    if (err) return sg_fail(SG_ERR_TIMEOUT, "batch: grid barrier wait expired");
    done_all = 1;
    for (int k = 0; k < b->nseq; ++k) done_all &= poll[k].done;
    if (b->graph_while) {        // persistent launches the WHILE node ran
      int most = 1;
      for (int k = 0; k < b->nseq; ++k) if (active[k] && poll[k].iter > most) most = poll[k].iter;
      sg_count_launches(most);
      // the last running system continues alone in its own iteration graph
      // (operator step + update over that system's grid only), which is cheaper
      // than persistent launches over the whole batch grid
      int left = -1, nleft = 0;
      for (int k = 0; k < b->nseq; ++k)
        if (active[k] && !poll[k].done) { left = k; ++nleft; }
      if (nleft == 1) {
        int rc = batch_solo(b, left, s);
        if (rc) return rc;
        const int before = poll[left].iter;
        SG_CUDA_TRY(cudaMemcpyAsync(&poll[left], &A.seq[left].st->iter, sizeof(PollS), cudaMemcpyDeviceToHost, s));
        SG_CUDA_TRY(cudaStreamSynchronize(s));
        sg_count_launches(2 * (poll[left].iter - before > 0 ? poll[left].iter - before : 1));
        done_all = 1;
        for (int k = 0; k < b->nseq; ++k) done_all &= poll[k].done;
      }
    }
    if (replays >= max_replays) break;
  }
  for (int k = 0; k < b->nseq; ++k) {
    if (iters) iters[k] = active[k] ? poll[k].iter : 0;
    if (active[k] && poll[k].status == PCG_BREAKDOWN) return sg_fail(SG_ERR_BREAKDOWN, "batch: PCG breakdown");
  }
  return SG_OK;
}

extern "C" int sg_batch_ir_solve(sg_batch_t b, const void* const* bvec, void* const* xvec, double tol, double inner_tol,
                                 int max_outer, int maxit_inner, int* outer_iters, int* inner_iters, double* relres,
                                 void* stream) {
  if (!b || !bvec || !xvec) return sg_fail(SG_ERR_INVALID, "batch_ir_solve: NULL argument");
  if (!(tol > 0.0) || !(inner_tol > 0.0) || max_outer < 0 || maxit_inner < 0)
    return sg_fail(SG_ERR_INVALID, "batch_ir_solve: bad tolerance or limit");
  cudaStream_t s = as_stream(stream);
  const int ns = b->nseq;
  for (int k = 0; k < ns; ++k) {
    if (!bvec[k] || !xvec[k] || !aligned16(bvec[k]) || !aligned16(xvec[k]))
      return sg_fail(SG_ERR_INVALID, "batch_ir_solve: vectors must be non-NULL and 16-byte aligned");
    const SemGeom& g = b->op64[k]->g;
    k_batch_mask<double><<<64, 256, 0, s>>>(static_cast<double*>(xvec[k]), g.nx, g.ny, g.nz);
    SG_LAUNCH_CHECK("k_batch_mask");
  }
  int active[SG_BATCH_MAX] = {0}, outer[SG_BATCH_MAX] = {0}, inner[SG_BATCH_MAX] = {0};
  double rel[SG_BATCH_MAX] = {0};
  PcgState* st = reinterpret_cast<PcgState*>(b->ws + b->off_state);
  double* partials = reinterpret_cast<double*>(b->ws + b->off_partials);
  for (int round = 0;; ++round) {
    // FP64 residual of every system still running
    int any = 0;
    for (int k = 0; k < ns; ++k) {
      if (round > 0 && !active[k]) continue;
      SemArgs<double> a{};
      a.x = static_cast<const double*>(xvec[k]);
      a.aux = static_cast<const double*>(bvec[k]);
      a.out = reinterpret_cast<double*>(b->ws + b->off_r64[k]);
      a.partials = partials; a.st = st + k; a.final_pass = 1;
      k_pcg_state_reset_counters<<<1, 32, 0, s>>>(st + k);
      SG_LAUNCH_CHECK("k_pcg_state_reset_counters");
      int rc = sg_sem_launch<double, 2>(b->op64[k]->g, a, s, 0);
      if (rc) return rc;
      PcgState hs;
      SG_CUDA_TRY(cudaMemcpyAsync(&hs, st + k, sizeof(PcgState), cudaMemcpyDeviceToHost, s));
      SG_CUDA_TRY(cudaStreamSynchronize(s));
      rel[k] = hs.bb > 0 ? std::sqrt(hs.rr_true / hs.bb) : std::sqrt(hs.rr_true);
      if (!std::isfinite(rel[k])) return sg_fail(SG_ERR_BREAKDOWN, "batch_ir_solve: non-finite residual");
      active[k] = (rel[k] > tol && outer[k] < max_outer) ? 1 : 0;
      any |= active[k];
      if (active[k]) {
        const int n = (int)b->op64[k]->n;
        k_batch_to_f32<<<16 * sg_num_sms(), 256, 0, s>>>(a.out, reinterpret_cast<float*>(b->ws + b->off_vec[k][6]), n);
        SG_LAUNCH_CHECK("k_batch_to_f32");
      }
    }
    if (!any) break;
    int it[SG_BATCH_MAX] = {0};
    BatchTol itol{};
    for (int k = 0; k < ns; ++k) itol.rel[k] = active[k] ? ir_inner_tol(inner_tol, tol, rel[k]) : inner_tol;
    int rc = batch_inner(b, active, itol, maxit_inner, it, s);
    if (rc) return rc;
    for (int k = 0; k < ns; ++k) {
      if (!active[k]) continue;
      inner[k] += it[k];
      outer[k] += 1;
      k_batch_add<<<16 * sg_num_sms(), 256, 0, s>>>(static_cast<double*>(xvec[k]),
                                                    reinterpret_cast<const float*>(b->ws + b->off_vec[k][0]),
                                                    (int)b->op64[k]->n);
      SG_LAUNCH_CHECK("k_batch_add");
    }
  }
  int status = SG_OK;
  for (int k = 0; k < ns; ++k) {
    if (outer_iters) outer_iters[k] = outer[k];
    if (inner_iters) inner_iters[k] = inner[k];
    if (relres) relres[k] = rel[k];
    if (rel[k] > tol) status = SG_NOT_CONVERGED;
  }
  if (status == SG_NOT_CONVERGED) sg_set_error("batch_ir_solve: maximum outer iteration count reached");
  return status;
}

// Autotuner: time a few persistent iterations for each candidate (z-chunk
// depth of the work items x CTAs per SM) on the current right-hand sides of
// all systems, keep the fastest.  Results (ms per iteration) are returned.
extern "C" int sg_batch_tune(sg_batch_t b, int* best_zl, int* best_blocks_per_sm, double* best_ms, void* stream) {
  if (!b) return sg_fail(SG_ERR_INVALID, "batch_tune: NULL handle");
  cudaStream_t s = as_stream(stream);
  int per_sm = 0;
  int rc = max_coresident(&per_sm);
  if (rc) return rc;
  const int zls[] = {1, 2, 3, 4};
  double best = 1e30;
  int bz = b->zl, bb = b->blocks_per_sm;
  int active[SG_BATCH_MAX];
  for (int k = 0; k < b->nseq; ++k) {
    active[k] = 1;
    // a deterministic non-trivial right-hand side: b = 1 on interior nodes
    const SemGeom& g = b->op32[k]->g;
    float* bv = reinterpret_cast<float*>(b->ws + b->off_vec[k][6]);
    k_convert_fill<<<16 * sg_num_sms(), 256, 0, s>>>(bv, (int)b->op32[k]->n);
    sg_count_launch();
    k_batch_mask<float><<<64, 256, 0, s>>>(bv, g.nx, g.ny, g.nz);
    sg_count_launch();
  }
  cudaEvent_t e0, e1;
  SG_CUDA_TRY(cudaEventCreate(&e0));
  SG_CUDA_TRY(cudaEventCreate(&e1));
  BatchArgs A = make_args(b);
  for (int zl : zls) {
    rc = build_items(b, zl, s);
    if (rc) break;
    for (int bps = 1; bps <= per_sm; ++bps) {
      b->blocks_per_sm = bps;
      b->nblocks = bps * sg_num_sms();
      A = make_args(b);
      int gx = 4 * sg_num_sms() / b->nseq;
      cudaMemcpyAsync(b->ws + b->off_active, active, sizeof(int) * b->nseq, cudaMemcpyHostToDevice, s);
      BatchTol none{};
      for (int k = 0; k < SG_BATCH_MAX; ++k) none.rel[k] = 1e-30;
      k_batch_init<<<dim3(gx > 0 ? gx : 1, b->nseq), 256, 0, s>>>(A, none, 1 << 30,
          reinterpret_cast<unsigned int*>(b->ws + b->off_counters), reinterpret_cast<const int*>(b->ws + b->off_active));
      sg_count_launch();
      for (int w = 0; w < 2; ++w) if ((rc = launch_iter(b, s))) break;
      cudaEventRecord(e0, s);
      const int reps = 6;
      for (int w = 0; w < reps && !rc; ++w) rc = launch_iter(b, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      if (rc) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      if (ms < best) { best = ms; bz = zl; bb = bps; }
    }
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->blocks_per_sm = bb;
  b->nblocks = bb * sg_num_sms();
  rc = build_items(b, bz, s);
  if (rc) return rc;
  if (b->graph_ready) { cudaGraphExecDestroy(b->graph); b->graph_ready = 0; }
  b->tuned = 1;
  if (best_zl) *best_zl = bz;
  if (best_blocks_per_sm) *best_blocks_per_sm = bb;
  if (best_ms) *best_ms = best;
  return SG_OK;
}

// ---------------------------------------------------------------- barrier self-test
// One cooperative launch that passes through the grid barrier twice.  With
// extra_blocks > 0 the barrier expects that many CTAs more than are launched,
// so its bounded wait must expire: the kernel records the expiry in the error
// word and returns normally, and the host reports SG_ERR_TIMEOUT.
__global__ void k_barrier_selftest(unsigned int* bar, int* err, unsigned int expect, long long spin_limit, int* passes) {
  grid_barrier(bar, err, expect, spin_limit);
  if (threadIdx.x == 0 && blockIdx.x == 0) atomicAdd(passes, 1);
  grid_barrier(bar, err, expect, spin_limit);
}

extern "C" int sg_selftest_barrier(int extra_blocks, long long spin_limit, void* scratch, void* stream) {
  if (!scratch || extra_blocks < 0 || spin_limit < 1) return sg_fail(SG_ERR_INVALID, "selftest_barrier: bad argument");
  cudaStream_t s = as_stream(stream);
  unsigned int* bar = static_cast<unsigned int*>(scratch);
  int* err = reinterpret_cast<int*>(bar + 2);
  int* passes = err + 1;
  SG_CUDA_TRY(cudaMemsetAsync(scratch, 0, 16, s));
  int blocks = sg_num_sms();
  unsigned int expect = (unsigned int)(blocks + extra_blocks);
  void* params[] = {&bar, &err, &expect, &spin_limit, &passes};
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelExC(&cfg, (const void*)k_barrier_selftest, params);
  sg_count_launch();
  if (e != cudaSuccess) return sg_fail(SG_ERR_CUDA, std::string("selftest_barrier launch: ") + cudaGetErrorString(e));
  int h[2] = {0, 0};
  SG_CUDA_TRY(cudaMemcpyAsync(h, err, sizeof(int) * 2, cudaMemcpyDeviceToHost, s));
  SG_CUDA_TRY(cudaStreamSynchronize(s));
  if (h[0]) return sg_fail(SG_ERR_TIMEOUT, "selftest_barrier: grid barrier wait expired");
  return SG_OK;
}
