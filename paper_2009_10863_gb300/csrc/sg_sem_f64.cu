// Explicit FP64 instantiations of the SEM operator kernel (all degrees, modes).
#include "sg_sem_launch.cuh"
template int sg_sem_launch<double, 0>(const SemGeom&, const SemArgs<double>&, cudaStream_t, int);
template int sg_sem_launch<double, 1>(const SemGeom&, const SemArgs<double>&, cudaStream_t, int);
template int sg_sem_launch<double, 2>(const SemGeom&, const SemArgs<double>&, cudaStream_t, int);
template int sg_sem_prepare<double, 1>(const SemGeom&);
