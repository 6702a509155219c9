// sg_sem_launch.cuh -- host-side dispatch of k_sem over (dtype, degree, mode).
#pragma once
#include <cstring>

#include "sg_sem_kernel.cuh"

// Element layers per CTA: enough CTAs for ~4 per SM, fewer layers means more
// restaging of the first plane and of the z-carry per chunk.
int sg_sem_layers(const SemGeom& g, int tex, int tey, int override_zl);

template <typename T, int P>
constexpr size_t sem_smem_bytes() {
  using TL = SemTile<P>;
  return sizeof(T) * ((size_t)TL::NPL * TL::PY * TL::template pitch<T>() +
                      (TL::template two_w<T>() ? 2 : 1) * (size_t)P * TL::TY * TL::TX);
}

// Dynamic shared-memory attribute of one instantiation (once per process; it
// is not a stream operation, so it is done before a launch is captured).
template <typename T, int P, int MODE>
int sg_sem_attr_p() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_sem<T, P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sem_smem_bytes<T, P>());
    if (e != cudaSuccess) return sg_fail(SG_ERR_CUDA, std::string("sem smem attribute: ") + cudaGetErrorString(e));
    attr_set = true;
  }
  return SG_OK;
}

template <typename T, int P, int MODE>
int sg_sem_launch_p(const SemGeom& g, const SemArgs<T>& a0, cudaStream_t s, int zl_override) {
  using TL = SemTile<P>;
  if (!g.tabs) return sg_fail(SG_ERR_STATE, "sem: the operator was created without a CUDA device");
  SemArgs<T> a = a0;
  a.zl = sg_sem_layers(g, TL::TEX, TL::TEY, zl_override);
  dim3 block(TL::TX, TL::TY, 1);
  dim3 grid((g.ex + TL::TEX - 1) / TL::TEX, (g.ey + TL::TEY - 1) / TL::TEY,
            (g.ez + a.zl - 1) / a.zl);
  const size_t smem = sem_smem_bytes<T, P>();
  int rc = sg_sem_attr_p<T, P, MODE>();
  if (rc) return rc;
  SemTabs<T, P> tb;                              // the coefficients, by value
  std::memcpy(&tb, g.htabs, sizeof(tb));
  k_sem<T, P, MODE><<<grid, block, smem, s>>>(g, a, tb);
  SG_LAUNCH_CHECK("k_sem");
  return SG_OK;
}

template <typename T, int MODE>
int sg_sem_launch(const SemGeom& g, const SemArgs<T>& a, cudaStream_t s, int zl_override = 0) {
  switch (g.p) {
    case 1: return sg_sem_launch_p<T, 1, MODE>(g, a, s, zl_override);
    case 2: return sg_sem_launch_p<T, 2, MODE>(g, a, s, zl_override);
    case 3: return sg_sem_launch_p<T, 3, MODE>(g, a, s, zl_override);
    case 4: return sg_sem_launch_p<T, 4, MODE>(g, a, s, zl_override);
    case 5: return sg_sem_launch_p<T, 5, MODE>(g, a, s, zl_override);
    case 6: return sg_sem_launch_p<T, 6, MODE>(g, a, s, zl_override);
    case 7: return sg_sem_launch_p<T, 7, MODE>(g, a, s, zl_override);
    case 8: return sg_sem_launch_p<T, 8, MODE>(g, a, s, zl_override);
    default: return sg_fail(SG_ERR_INVALID, "degree p out of range");
  }
}

template <typename T, int MODE>
int sg_sem_prepare(const SemGeom& g) {
  switch (g.p) {
    case 1: return sg_sem_attr_p<T, 1, MODE>();
    case 2: return sg_sem_attr_p<T, 2, MODE>();
    case 3: return sg_sem_attr_p<T, 3, MODE>();
    case 4: return sg_sem_attr_p<T, 4, MODE>();
    case 5: return sg_sem_attr_p<T, 5, MODE>();
    case 6: return sg_sem_attr_p<T, 6, MODE>();
    case 7: return sg_sem_attr_p<T, 7, MODE>();
    case 8: return sg_sem_attr_p<T, 8, MODE>();
    default: return sg_fail(SG_ERR_INVALID, "degree p out of range");
  }
}

// explicit instantiations live in sg_sem_f64.cu / sg_sem_f32.cu
extern template int sg_sem_launch<double, 0>(const SemGeom&, const SemArgs<double>&, cudaStream_t, int);
extern template int sg_sem_launch<double, 1>(const SemGeom&, const SemArgs<double>&, cudaStream_t, int);
extern template int sg_sem_launch<double, 2>(const SemGeom&, const SemArgs<double>&, cudaStream_t, int);
extern template int sg_sem_launch<float, 0>(const SemGeom&, const SemArgs<float>&, cudaStream_t, int);
extern template int sg_sem_launch<float, 1>(const SemGeom&, const SemArgs<float>&, cudaStream_t, int);
extern template int sg_sem_launch<float, 2>(const SemGeom&, const SemArgs<float>&, cudaStream_t, int);
extern template int sg_sem_prepare<double, 1>(const SemGeom&);
extern template int sg_sem_prepare<float, 1>(const SemGeom&);
