// probe.cu -- FMA probes of the GPU (measurement utilities, not part of the
// scheme).  qnsch_fma_probe gives the FP64 peak that bench.py divides the FP64
// kernels' achieved rate by: each thread runs eight independent FMA chains, so
// the pipe, not the dependent-instruction latency, sets the rate.
// qnsch_fp64_issue_probe gives the SM cycles one warp-wide FP64 FMA holds a
// sub-partition for, as a function of the active lanes and of the independent
// chains per lane: the cost model behind the solver's launch shapes.
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

// One block per SM.  The first `active` lanes of every warp run `CH`
// independent chains of 16 x iters FMAs; thread 0 records the block's elapsed
// SM cycles between two barriers.
template <typename T, int CH>
__global__ void k_issue_probe(T* out, long long* cycles, int iters, int active, T b) {
  T a[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) a[c] = T(threadIdx.x) * T(1e-3) + T(c);
  const T m = T(0.999);
  __syncthreads();
  const long long t0 = clock64();
  if ((int)(threadIdx.x & 31) < active) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
#pragma unroll
        for (int c = 0; c < CH; ++c) a[c] = fma(a[c], m, b);
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
  T s = T(0);
#pragma unroll
  for (int c = 0; c < CH; ++c) s += a[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int run_issue_probe(int warps, int active, int chains, int iters, double* cpi) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ENODEV;
  }
  const int threads = 32 * warps;
  double* out = nullptr;
  long long* cyc = nullptr;
  if (cudaMalloc(&out, (size_t)sms * threads * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&cyc, (size_t)sms * sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(out);
    return QNSCH_ENOMEM;
  }
  long long* host = new long long[sms];
  long long best = -1;
  int rc = QNSCH_OK;
  for (int k = 0; k < 4 && rc == QNSCH_OK; ++k) {  // first launch warms up
    switch (chains) {
      case 1: k_issue_probe<double, 1><<<sms, threads>>>(out, cyc, iters, active, 1e-3); break;
      case 2: k_issue_probe<double, 2><<<sms, threads>>>(out, cyc, iters, active, 1e-3); break;
      case 4: k_issue_probe<double, 4><<<sms, threads>>>(out, cyc, iters, active, 1e-3); break;
      default: k_issue_probe<double, 8><<<sms, threads>>>(out, cyc, iters, active, 1e-3); break;
    }
    if (cudaMemcpy(host, cyc, (size_t)sms * sizeof(long long), cudaMemcpyDeviceToHost) !=
        cudaSuccess) {
      cudaGetLastError();
      rc = QNSCH_ECUDA;
      break;
    }
    if (k == 0) continue;
    long long worst = 0;
    for (int b = 0; b < sms; ++b) worst = host[b] > worst ? host[b] : worst;
    if (best < 0 || worst < best) best = worst;
  }
  if (rc == QNSCH_OK) {
    const int per_sp = (warps + 3) / 4;  // warps on the busiest of 4 sub-partitions
    *cpi = (double)best / (16.0 * chains * (double)iters * per_sp);
  }
  delete[] host;
  cudaFree(out);
  cudaFree(cyc);
  return rc;
}

}  // namespace

extern "C" int qnsch_fp64_issue_probe(int warps_per_block, int active_lanes, int chains, int iters,
                                      double* cycles_per_instr) {
  if (!cycles_per_instr || warps_per_block < 1 || warps_per_block > 32 || active_lanes < 1 ||
      active_lanes > 32 || !(chains == 1 || chains == 2 || chains == 4 || chains == 8) ||
      iters < 1 || iters > (1 << 20))
    return QNSCH_EINVAL;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return QNSCH_ENODEV;
  }
  return run_issue_probe(warps_per_block, active_lanes, chains, iters, cycles_per_instr);
}

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
