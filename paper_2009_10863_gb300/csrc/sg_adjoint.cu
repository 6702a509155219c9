// sg_adjoint.cu -- vector kernels of a time-stepped Helmholtz sequence and of
// its reverse-time adjoint (FP64).
//
// Sequence (implicit time stepping, Sec. 5.2; Helmholtz systems of Eq.
// VelocityEqn): A x_k = M (lam x_{k-1} + f_k), A = K + lam M, with K the SEM
// stiffness and M the (diagonal) GLL mass matrix of Sec. 5.1.  Loss
// L = sum_k ||x_k - x*_k||^2.  Adjoint (A, M symmetric), backward in time:
// A g_k = 2 (x_k - x*_k) + lam M g_{k+1}; dL/df_k = M g_k,
// dL/dlam = sum_k g_k^T M (x_{k-1} - x_k).  The solves use sg_pcg_solve; the
// kernels here build the right-hand sides and accumulate loss and gradient
// terms.  Reductions are deterministic (per-block partials summed in block
// order by the last block, which adds the total to a device accumulator).
#include "sg_sem_launch.cuh"

namespace {
constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
int adj_blocks(int64_t n) {
  int64_t b = (n + 255) / 256, cap = 8LL * sg_num_sms();
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}
struct AdjWs { double* partials; unsigned int* counter; };
AdjWs adj_ws(void* ws) {
  AdjWs w;
  w.counter = reinterpret_cast<unsigned int*>(ws);
  w.partials = reinterpret_cast<double*>(static_cast<unsigned char*>(ws) + kAlign);
  return w;
}
}

// GLL mass weight of global node i (0 on Dirichlet nodes).
__device__ __forceinline__ double mass_w(const SemGeom& g, const FastDiv& dnx, const FastDiv& dnxy, int i, double J) {
  const uint32_t k = dnxy.div((uint32_t)i);
  const uint32_t rem = (uint32_t)i - k * dnxy.d;
  const uint32_t j = dnx.div(rem);
  const uint32_t ii = rem - j * dnx.d;
  if (ii == 0 || j == 0 || k == 0 || (int)ii >= g.nx - 1 || (int)j >= g.ny - 1 || (int)k >= g.nz - 1) return 0.0;
  return J * g.wl[ii % g.p] * g.wl[j % g.p] * g.wl[k % g.p];
}

__global__ void k_mass_rhs(const SemGeom g, FastDiv dnx, FastDiv dnxy, int n, double J, double a,
                           const double* __restrict__ x, const double* __restrict__ f, double* __restrict__ rhs) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double w = mass_w(g, dnx, dnxy, i, J);
    double v = f ? f[i] : 0.0;
    if (x) v += a * x[i];
    rhs[i] = w * v;
  }
}

__global__ void k_adj_rhs(const SemGeom g, FastDiv dnx, FastDiv dnxy, int n, double J, double c,
                          const double* __restrict__ x, const double* __restrict__ xs, double a,
                          const double* __restrict__ gn, double* __restrict__ rhs) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double w = mass_w(g, dnx, dnxy, i, J);
    double v = (w != 0.0) ? c * (x[i] - xs[i]) : 0.0;
    if (gn) v += a * w * gn[i];
    rhs[i] = v;
  }
}

// out = M g (may be NULL); acc[0] += g^T M (xprev - x)   (xprev NULL = 0)
__global__ void __launch_bounds__(256) k_adj_accum(const SemGeom g, FastDiv dnx, FastDiv dnxy, int n, double J,
                                                   const double* __restrict__ gv, const double* __restrict__ xprev,
                                                   const double* __restrict__ x, double* __restrict__ out,
                                                   double* partials, unsigned int* counter, double* acc) {
  __shared__ double sred[32];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double w = mass_w(g, dnx, dnxy, i, J);
    const double mg = w * gv[i];
    if (out) out[i] = mg;
    s += mg * ((xprev ? xprev[i] : 0.0) - x[i]);
  }
  double v[1] = {s}, tot[1];
  if (grid_reduce_last<1>(v, partials, counter, sred, tot))
    if (threadIdx.x == 0) acc[0] += tot[0];
}

// acc[0] += sum over interior nodes of (x - xs)^2
__global__ void __launch_bounds__(256) k_sqdiff_accum(const SemGeom g, FastDiv dnx, FastDiv dnxy, int n,
                                                      const double* __restrict__ x, const double* __restrict__ xs,
                                                      double* partials, unsigned int* counter, double* acc) {
  __shared__ double sred[32];
  double s = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double w = mass_w(g, dnx, dnxy, i, 1.0);
    const double d = (w != 0.0) ? x[i] - xs[i] : 0.0;
    s += d * d;
  }
  double v[1] = {s}, tot[1];
  if (grid_reduce_last<1>(v, partials, counter, sred, tot))
    if (threadIdx.x == 0) acc[0] += tot[0];
}

static double mass_scale(sg_op_t op) {
  return (1.0 / op->g.ex) * (1.0 / op->g.ey) * (1.0 / op->g.ez) / 8.0;
}

static int check_op64(sg_op_t op, const char* who) {
  if (!op) return sg_fail(SG_ERR_INVALID, std::string(who) + ": NULL operator");
  if (op->dtype != SG_F64) return sg_fail(SG_ERR_INVALID, std::string(who) + ": FP64 operator required");
  return SG_OK;
}

extern "C" size_t sg_seq_workspace_bytes(sg_op_t op) {
  if (!op) return 0;
  return kAlign + align_up(sizeof(double) * (size_t)adj_blocks(op->n));
}

extern "C" int sg_mass_rhs(sg_op_t op, double a, const void* x, const void* f, void* rhs, void* stream) {
  int rc = check_op64(op, "mass_rhs");
  if (rc) return rc;
  if (!rhs || (!x && !f)) return sg_fail(SG_ERR_INVALID, "mass_rhs: NULL argument");
  const int n = (int)op->n;
  k_mass_rhs<<<adj_blocks(n), 256, 0, as_stream(stream)>>>(op->g, op->div_nx, op->div_nxy, n, mass_scale(op), a,
                                                           static_cast<const double*>(x), static_cast<const double*>(f),
                                                           static_cast<double*>(rhs));
  SG_LAUNCH_CHECK("k_mass_rhs");
  return SG_OK;
}

extern "C" int sg_adjoint_rhs(sg_op_t op, double c, const void* x, const void* xs, double a, const void* gnext,
                              void* rhs, void* stream) {
  int rc = check_op64(op, "adjoint_rhs");
  if (rc) return rc;
  if (!x || !xs || !rhs) return sg_fail(SG_ERR_INVALID, "adjoint_rhs: NULL argument");
  const int n = (int)op->n;
  k_adj_rhs<<<adj_blocks(n), 256, 0, as_stream(stream)>>>(op->g, op->div_nx, op->div_nxy, n, mass_scale(op), c,
                                                          static_cast<const double*>(x), static_cast<const double*>(xs), a,
                                                          static_cast<const double*>(gnext), static_cast<double*>(rhs));
  SG_LAUNCH_CHECK("k_adj_rhs");
  return SG_OK;
}

extern "C" int sg_adjoint_accum(sg_op_t op, const void* g, const void* xprev, const void* x, void* mg, double* acc,
                                void* workspace, void* stream) {
  int rc = check_op64(op, "adjoint_accum");
  if (rc) return rc;
  if (!g || !x || !acc || !workspace) return sg_fail(SG_ERR_INVALID, "adjoint_accum: NULL argument");
  const int n = (int)op->n;
  AdjWs w = adj_ws(workspace);
  k_adj_accum<<<adj_blocks(n), 256, 0, as_stream(stream)>>>(op->g, op->div_nx, op->div_nxy, n, mass_scale(op),
                                                            static_cast<const double*>(g), static_cast<const double*>(xprev),
                                                            static_cast<const double*>(x), static_cast<double*>(mg),
                                                            w.partials, w.counter, acc);
  SG_LAUNCH_CHECK("k_adj_accum");
  return SG_OK;
}

extern "C" int sg_sqdiff_accum(sg_op_t op, const void* x, const void* xs, double* acc, void* workspace, void* stream) {
  int rc = check_op64(op, "sqdiff_accum");
  if (rc) return rc;
  if (!x || !xs || !acc || !workspace) return sg_fail(SG_ERR_INVALID, "sqdiff_accum: NULL argument");
  const int n = (int)op->n;
  AdjWs w = adj_ws(workspace);
  k_sqdiff_accum<<<adj_blocks(n), 256, 0, as_stream(stream)>>>(op->g, op->div_nx, op->div_nxy, n,
                                                               static_cast<const double*>(x), static_cast<const double*>(xs),
                                                               w.partials, w.counter, acc);
  SG_LAUNCH_CHECK("k_sqdiff_accum");
  return SG_OK;
}
