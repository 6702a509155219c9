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

// Deterministic block sum of NV values per thread (fixed shuffle tree, then a
// fixed-order combine of warp results).  Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /* >= 32*NV */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int tl = tid & 31, tw = tid >> 5;
  (void)lane; (void)warp;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (tl == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[k * 32 + tw] = v[k];
  }
  __syncthreads();
  if (tw == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double a = (tl < nwarps) ? smem[k * 32 + tl] : 0.0;
      v[k] = warp_sum(a);
    }
  }
  __syncthreads();
}

// Deterministic block sum of two values per thread with half the FP64
// additions of two separate shuffle trees: one exchange at distance 16 leaves
// partial sums of a in lanes 0-15 and of b in lanes 16-31, and four more rounds
// reduce one value per lane.  Blocks of at most 512 threads.  Results valid in
// thread 0 (a and b).
__device__ __forceinline__ void block_sum2(double& a, double& b, double* smem /* >= 64 */) {
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nwarps = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
  const int tl = tid & 31, tw = tid >> 5;
  const bool hi = (tl & 16) != 0;
  double keep = hi ? b : a;
  const double give = hi ? a : b;
  keep += __shfl_xor_sync(0xffffffffu, give, 16);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  __syncthreads();
  if (tl == 0) smem[tw] = keep;             // warp sum of a
  if (tl == 16) smem[32 + tw] = keep;       // warp sum of b
  __syncthreads();
  if (tw == 0) {
    const int w = tl & 15;
    double x = (w < nwarps) ? smem[(hi ? 32 : 0) + w] : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const double xb = __shfl_sync(0xffffffffu, x, 16);
    if (tl == 0) { a = x; b = xb; }
  }
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ void block_sum_any(double (&v)[NV], double* smem) {
  if constexpr (NV == 2) block_sum2(v[0], v[1], smem);
  else block_sum<NV>(v, smem);
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
  block_sum_any<NV>(v, smem);
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
  block_sum_any<NV>(acc, smem);
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
