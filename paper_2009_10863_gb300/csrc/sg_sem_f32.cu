// Explicit FP32 instantiations of the SEM operator kernel (all degrees, modes).
#include "sg_sem_launch.cuh"
template int sg_sem_launch<float, 0>(const SemGeom&, const SemArgs<float>&, cudaStream_t, int);
template int sg_sem_launch<float, 1>(const SemGeom&, const SemArgs<float>&, cudaStream_t, int);
template int sg_sem_launch<float, 2>(const SemGeom&, const SemArgs<float>&, cudaStream_t, int);
template int sg_sem_prepare<float, 1>(const SemGeom&);
