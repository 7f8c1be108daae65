// probe.cu -- FMA throughput probe of the GPU (a measurement utility, not part
// of the scheme): the FP64 figure is the peak that bench.py divides the FP64
// kernels' achieved rate by.  Each thread runs eight independent FMA chains,
// so the pipe, not the dependent-instruction latency, sets the rate.
#include <cuda_runtime.h>

#include "qnsch.h"

namespace {

template <typename T>
__global__ void k_fma_probe(T* out, int iters, T b) {
  T a0 = T(threadIdx.x) * T(1e-3), a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
  T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
  const T c = T(0.999);  // a -> a c + b stays bounded: a tends to b / (1 - c)
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      a0 = fma(a0, c, b);
      a1 = fma(a1, c, b);
      a2 = fma(a2, c, b);
      a3 = fma(a3, c, b);
      a4 = fma(a4, c, b);
      a5 = fma(a5, c, b);
      a6 = fma(a6, c, b);
      a7 = fma(a7, c, b);
    }
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

template <typename T>
int run_probe(int blocks_per_sm, int iters, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ENODEV;
  }
  const int threads = 256, blocks = sms * blocks_per_sm;
  T* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int k = 0; k < 3; ++k) k_fma_probe<T><<<blocks, threads>>>(out, iters, T(1e-3));
  cudaEventRecord(e0);
  const int timed = 5;
  for (int k = 0; k < timed; ++k) k_fma_probe<T><<<blocks, threads>>>(out, iters, T(1e-3));
  cudaEventRecord(e1);
  int rc = QNSCH_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
      !(ms > 0.f)) {
    cudaGetLastError();
    rc = QNSCH_ECUDA;
  } else {
    double flops = 2.0 * 8.0 * 16.0 * iters * (double)blocks * threads * timed;
    *tflops = flops / (ms * 1e-3) / 1e12;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace

extern "C" int qnsch_fma_probe(int fp64, int blocks_per_sm, int iters, double* tflops) {
  if (!tflops || blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || iters > (1 << 24))
    return QNSCH_EINVAL;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return QNSCH_ENODEV;
  }
  return fp64 ? run_probe<double>(blocks_per_sm, iters, tflops)
              : run_probe<float>(blocks_per_sm, iters, tflops);
}
