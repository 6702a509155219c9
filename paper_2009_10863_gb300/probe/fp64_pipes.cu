// fp64_pipes.cu -- throughput of the two FP64 paths of the SM: DFMA on the
// CUDA cores and the FP64 tensor-core MMA (mma.sync m8n8k4 / m16n8k16 .f64),
// each alone and both interleaved in one instruction stream.  The element
// contractions of the SEM operator are small dense FP64 products; this
// program measures which path can execute them faster.
//
// Every thread keeps its operands in registers and writes one double to
// out[global thread index]; there is no other memory access.
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ void mma_m8n8k4(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1) : "d"(a), "d"(b));
}

__device__ __forceinline__ void mma_m16n8k16(double (&c)[4], const double (&a)[8], const double (&b)[4]) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
               "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
               : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
               : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
                 "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

// MODE 0: 8 independent DFMA chains; 1: 4 independent m8n8k4 MMAs;
// 2: both per iteration; 3: 4 independent m16n8k16 MMAs.
template <int MODE>
__global__ void k_pipe(double* out, int iters, double s) {
  const double a = 1.0 + 1e-9 * threadIdx.x, b = 1.0 - 1e-9 * threadIdx.x;
  double f[8], acc[8], c[4][4], A[8], B[4];
#pragma unroll
  for (int k = 0; k < 8; ++k) { f[k] = s * (k + 1); acc[k] = s * k; A[k] = a * (k + 1); }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    B[k] = b * (k + 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) c[k][j] = 0.0;
  }
  for (int i = 0; i < iters; ++i) {
    if (MODE == 0 || MODE == 2) {
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = fma(f[k], a, b);
    }
    if (MODE == 1 || MODE == 2) {
#pragma unroll
      for (int k = 0; k < 4; ++k) mma_m8n8k4(acc[2 * k], acc[2 * k + 1], a, b);
    }
    if (MODE == 3) {
#pragma unroll
      for (int k = 0; k < 4; ++k) mma_m16n8k16(c[k], A, B);
    }
  }
  double r = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) r += acc[k] + f[k];
#pragma unroll
  for (int k = 0; k < 4; ++k) r += c[k][0] + c[k][1] + c[k][2] + c[k][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { \
  printf("CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); return 1; } } while (0)

int main() {
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
  const int threads = 256, blocks = 4 * sms, iters = 4096;
  double* out = nullptr;
  CK(cudaMalloc(&out, sizeof(double) * threads * blocks));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const char* names[4] = {"DFMA x8 (CUDA cores)", "MMA m8n8k4 x4", "DFMA x8 + MMA m8n8k4 x4", "MMA m16n8k16 x4"};
  const double warps = (double)blocks * threads / 32.0;
  printf("%d SMs, %d blocks x %d threads, %d iterations\n", sms, blocks, threads, iters);
  for (int mode = 0; mode < 4; ++mode) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      CK(cudaEventRecord(e0));
      if (mode == 0) k_pipe<0><<<blocks, threads>>>(out, iters, 1e-3);
      if (mode == 1) k_pipe<1><<<blocks, threads>>>(out, iters, 1e-3);
      if (mode == 2) k_pipe<2><<<blocks, threads>>>(out, iters, 1e-3);
      if (mode == 3) k_pipe<3><<<blocks, threads>>>(out, iters, 1e-3);
      CK(cudaGetLastError());
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && ms < best) best = ms;
    }
    const double fl_fma = (mode == 0 || mode == 2) ? (double)blocks * threads * iters * 8 * 2 : 0.0;
    const double fl_mma = (mode == 1 || mode == 2) ? warps * iters * 4 * 512.0
                        : (mode == 3 ? warps * iters * 4 * 4096.0 : 0.0);
    printf("%-26s %9.3f ms   DFMA %7.1f GFLOP/s   MMA %7.1f GFLOP/s   total %7.1f GFLOP/s\n", names[mode], best,
           fl_fma / best * 1e-6, fl_mma / best * 1e-6, (fl_fma + fl_mma) / best * 1e-6);
  }
  CK(cudaFree(out));
  return 0;
}
