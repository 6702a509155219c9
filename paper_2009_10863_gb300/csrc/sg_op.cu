// sg_op.cu -- operator handle, sg_sem_apply, diagonal, errors and kernel timing.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sg_sem_launch.cuh"

namespace sgb {
void gll(int p, double* x, double* w);
void derivative(int p, const double* x, double* D);
void stiffness(int p, const double* D, const double* w, double* K);
}

// ---------------------------------------------------------------- errors
static thread_local std::string g_err;
void sg_set_error(const std::string& msg) { g_err = msg; }
int sg_fail(int code, const std::string& msg) { g_err = msg; return code; }
extern "C" const char* sg_last_error(void) { return g_err.c_str(); }
extern "C" int sg_version(void) { return 1; }

static std::atomic<long long> g_launches{0};
void sg_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void sg_count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
extern "C" long long sg_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int sg_num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// ---------------------------------------------------------------- kernel timing
namespace {
struct ProfEntry { cudaEvent_t a, b; int id; };
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfEntry> g_prof_pending;
double g_prof_ms[PROF_N];
long long g_prof_count[PROF_N];
std::vector<cudaEvent_t> g_prof_pool;

cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) { cudaEvent_t e = g_prof_pool.back(); g_prof_pool.pop_back(); return e; }
  cudaEvent_t e; cudaEventCreate(&e); return e;
}
void prof_drain() {   // caller holds the lock; synchronises on pending events
  for (auto& p : g_prof_pending) {
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    g_prof_ms[p.id] += ms;
    g_prof_count[p.id] += 1;
    g_prof_pool.push_back(p.a);
    g_prof_pool.push_back(p.b);
  }
  g_prof_pending.clear();
}
thread_local cudaEvent_t t_open_event = nullptr;
}  // namespace

ProfScope::ProfScope(int id_, cudaStream_t s_) : id(id_), s(s_), active(0) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  t_open_event = prof_event();
  cudaEventRecord(t_open_event, s);
  active = 1;
}
ProfScope::~ProfScope() {
  if (!active) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t b = prof_event();
  cudaEventRecord(b, s);
  g_prof_pending.push_back({t_open_event, b, id});
  if (g_prof_pending.size() > 4096) prof_drain();
}

extern "C" int sg_profile_enable(int on) { g_prof_on = (on != 0); return SG_OK; }
bool sg_profiling_on() { return g_prof_on; }
extern "C" int sg_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain();
  for (int i = 0; i < PROF_N; ++i) { g_prof_ms[i] = 0.0; g_prof_count[i] = 0; }
  return SG_OK;
}
extern "C" int sg_profile_read(int id, double* total_ms, long long* launches) {
  if (id < 0 || id >= PROF_N) return sg_fail(SG_ERR_INVALID, "profile id out of range");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_drain();
  if (total_ms) *total_ms = g_prof_ms[id];
  if (launches) *launches = g_prof_count[id];
  return SG_OK;
}

// ---------------------------------------------------------------- operator
int sg_sem_layers(const SemGeom& g, int tex, int tey, int override_zl) {
  if (override_zl <= 0) override_zl = g.zl;
  if (override_zl > 0) return override_zl < g.ez ? override_zl : g.ez;
  const long nxy = (long)((g.ex + tex - 1) / tex) * ((g.ey + tey - 1) / tey);
  const long want = 8L * sg_num_sms();           // CTAs to aim for (several waves)
  long zl = (nxy * g.ez) / want;
  if (zl < 1) zl = 1;
  if (zl > g.ez) zl = g.ez;
  const long nchunks = (g.ez + zl - 1) / zl;     // balance: chunks differ by <= 1 layer
  zl = (g.ez + nchunks - 1) / nchunks;
  return (int)zl;
}

static void build_geom(sg_op_s* op) {
  SemGeom& g = op->g;
  const int p = g.p;
  const double hx = 1.0 / g.ex, hy = 1.0 / g.ey, hz = 1.0 / g.ez;
  double D[(SG_PMAX + 1) * (SG_PMAX + 1)], K[(SG_PMAX + 1) * (SG_PMAX + 1)];
  sgb::gll(p, op->nodes, op->weights);
  sgb::derivative(p, op->nodes, D);
  sgb::stiffness(p, D, op->weights, K);
  const double* w = op->weights;
  const int n1 = p + 1;
  // direction scales: J (2/h_dir)^2 with J = hx hy hz / 8
  const double adir[3] = {hy * hz / (2.0 * hx), hx * hz / (2.0 * hy), hx * hy / (2.0 * hz)};
  const double wsh = w[0] + w[p];
  std::memset(g.C, 0, sizeof(g.C));
  std::memset(g.dg, 0, sizeof(g.dg));
  for (int d = 0; d < 3; ++d) {
    for (int a = 0; a <= p; ++a) {
      const double wr = (a == 0 || a == p) ? wsh : w[a];
      for (int l = 0; l <= p; ++l) g.C[d][a][l] = adir[d] * K[a * n1 + l] / wr;
    }
    g.dg[d][0] = adir[d] * (K[0] + K[p * n1 + p]) / wsh;
    for (int a = 1; a < p; ++a) g.dg[d][a] = adir[d] * K[a * n1 + a] / w[a];
  }
  for (int a = 0; a <= p; ++a) g.wl[a] = (a == 0) ? wsh : w[a];
  for (int d = 0; d < 3; ++d) g.adir[d] = adir[d];
  g.cm = op->lambda * hx * hy * hz / 8.0;
}

// The operator kernel's coefficients (SemTabs: even-odd tables and weights),
// built in FP64 on the host and rounded to the operator's dtype.  The host
// copy is passed by value to every operator launch; the device copy serves
// the batched kernel's shared-memory tables.
template <typename T, int P>
static void fill_tables(const SemGeom& g, std::vector<unsigned char>& buf) {
  buf.assign(sizeof(SemTabs<T, P>), 0);
  sem_tables<T, P>(g, *reinterpret_cast<SemTabs<T, P>*>(buf.data()));
}

template <typename T>
static void fill_tables_p(const SemGeom& g, std::vector<unsigned char>& buf) {
  switch (g.p) {
    case 1: fill_tables<T, 1>(g, buf); break;
    case 2: fill_tables<T, 2>(g, buf); break;
    case 3: fill_tables<T, 3>(g, buf); break;
    case 4: fill_tables<T, 4>(g, buf); break;
    case 5: fill_tables<T, 5>(g, buf); break;
    case 6: fill_tables<T, 6>(g, buf); break;
    case 7: fill_tables<T, 7>(g, buf); break;
    default: fill_tables<T, 8>(g, buf); break;
  }
}

static int upload_tables(sg_op_s* op) {
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    // a host without a CUDA device: nothing can be launched, the handle still
    // answers the host queries (size, GLL nodes); launches refuse it
    cudaGetLastError();
    return SG_OK;
  }
  std::vector<unsigned char> buf;
  if (op->dtype == SG_F64) fill_tables_p<double>(op->g, buf);
  else fill_tables_p<float>(op->g, buf);
  if (buf.size() > sizeof(op->htabs)) return sg_fail(SG_ERR_INVALID, "op_create: coefficient tables too large");
  std::memcpy(op->htabs, buf.data(), buf.size());
  op->g.htabs = op->htabs;
  cudaError_t e = cudaMalloc(&op->d_tabs, buf.size());
  if (e != cudaSuccess) {
    op->d_tabs = nullptr;
    return sg_fail(SG_ERR_CUDA, std::string("op_create: table allocation: ") + cudaGetErrorString(e));
  }
  e = cudaMemcpy(op->d_tabs, buf.data(), buf.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(op->d_tabs);
    op->d_tabs = nullptr;
    return sg_fail(SG_ERR_CUDA, std::string("op_create: table upload: ") + cudaGetErrorString(e));
  }
  op->g.tabs = op->d_tabs;
  return SG_OK;
}

extern "C" int sg_op_create(sg_op_t* out, int ex, int ey, int ez, int p, double lambda, int dtype) {
  if (!out) return sg_fail(SG_ERR_INVALID, "op_create: NULL output handle");
  *out = nullptr;
  if (ex < 1 || ey < 1 || ez < 1) return sg_fail(SG_ERR_INVALID, "op_create: element counts must be >= 1");
  if (p < 1 || p > SG_PMAX) return sg_fail(SG_ERR_INVALID, "op_create: degree p must be in [1, 8]");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return sg_fail(SG_ERR_INVALID, "op_create: lambda must be finite and >= 0");
  if (dtype != SG_F64 && dtype != SG_F32) return sg_fail(SG_ERR_INVALID, "op_create: dtype must be SG_F64 or SG_F32");
  const long long nx = (long long)p * ex + 1, ny = (long long)p * ey + 1, nz = (long long)p * ez + 1;
  const long long n = nx * ny * nz;
  if (n >= (1LL << 31)) return sg_fail(SG_ERR_INVALID, "op_create: more than 2^31 - 1 nodes");
  sg_op_s* op = new sg_op_s();
  op->dtype = dtype;
  op->lambda = lambda;
  op->n = n;
  op->g.nx = (int)nx; op->g.ny = (int)ny; op->g.nz = (int)nz;
  op->g.ex = ex; op->g.ey = ey; op->g.ez = ez; op->g.p = p;
  build_geom(op);
  op->div_nx = FastDiv((uint32_t)nx);
  op->div_nxy = FastDiv((uint32_t)(nx * ny));
  // host self-check of the invariant-divisor division on a spread of values
  for (uint32_t t = 0; t < 4096; ++t) {
    uint32_t v = (uint32_t)(((uint64_t)t * 2654435761u) % (uint64_t)n);
    if (op->div_nx.div_host(v) != v / (uint32_t)nx || op->div_nxy.div_host(v) != v / (uint32_t)(nx * ny)) {
      delete op;
      return sg_fail(SG_ERR_INVALID, "op_create: internal divisor check failed");
    }
  }
  cudaGetDevice(&op->device);
  if (int rc = upload_tables(op)) {
    delete op;
    return rc;
  }
  static std::atomic<unsigned long long> next_uid{1};
  op->uid = next_uid.fetch_add(1);
  *out = op;
  return SG_OK;
}

extern "C" int sg_op_destroy(sg_op_t op) {
  if (op) {
    sg_pcg_release(op);
    if (op->d_tabs) cudaFree(op->d_tabs);
  }
  delete op;
  return SG_OK;
}

extern "C" int64_t sg_op_size(sg_op_t op) { return op ? op->n : -1; }

extern "C" int sg_op_set_layers(sg_op_t op, int zl) {
  if (!op) return sg_fail(SG_ERR_INVALID, "op_set_layers: NULL handle");
  if (zl < 0) return sg_fail(SG_ERR_INVALID, "op_set_layers: zl must be >= 0");
  op->g.zl = zl;
  sg_pcg_release(op);   // cached graphs hold the old launch shape
  return SG_OK;
}

extern "C" int sg_op_gll(sg_op_t op, double* nodes, double* weights) {
  if (!op) return sg_fail(SG_ERR_INVALID, "op_gll: NULL handle");
  for (int i = 0; i <= op->g.p; ++i) {
    if (nodes) nodes[i] = op->nodes[i];
    if (weights) weights[i] = op->weights[i];
  }
  return SG_OK;
}

extern "C" int sg_sem_apply(sg_op_t op, const void* x, void* y, void* stream) {
  if (!op || !x || !y) return sg_fail(SG_ERR_INVALID, "sem_apply: NULL argument");
  if (x == y) return sg_fail(SG_ERR_INVALID, "sem_apply: x and y must not alias");
  cudaStream_t s = as_stream(stream);
  ProfScope ps(PROF_SEM, s);
  if (op->dtype == SG_F64) {
    SemArgs<double> a{};
    a.x = static_cast<const double*>(x);
    a.out = static_cast<double*>(y);
    return sg_sem_launch<double, 0>(op->g, a, s, 0);
  }
  SemArgs<float> a{};
  a.x = static_cast<const float*>(x);
  a.out = static_cast<float*>(y);
  return sg_sem_launch<float, 0>(op->g, a, s, 0);
}

// diag(A) (inverse = 0) or 1/diag(A) (inverse = 1); 1 on Dirichlet nodes.
template <typename T>
__global__ void k_diag(const SemGeom g, FastDiv dnx, FastDiv dnxy, int n, int inverse, T* out) {
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
    out[i] = (T)(inverse ? 1.0 / v : v);
  }
}

int sg_op_diag_launch(sg_op_t op, void* out, int inverse, cudaStream_t s) {
  const int n = (int)op->n;
  const int threads = 256;
  int blocks = (n + threads - 1) / threads;
  if (blocks > 16 * sg_num_sms()) blocks = 16 * sg_num_sms();
  if (op->dtype == SG_F64)
    k_diag<double><<<blocks, threads, 0, s>>>(op->g, op->div_nx, op->div_nxy, n, inverse, static_cast<double*>(out));
  else
    k_diag<float><<<blocks, threads, 0, s>>>(op->g, op->div_nx, op->div_nxy, n, inverse, static_cast<float*>(out));
  SG_LAUNCH_CHECK("k_diag");
  return SG_OK;
}

extern "C" int sg_op_diagonal(sg_op_t op, void* diag, void* stream) {
  if (!op || !diag) return sg_fail(SG_ERR_INVALID, "op_diagonal: NULL argument");
  return sg_op_diag_launch(op, diag, 0, as_stream(stream));
}
