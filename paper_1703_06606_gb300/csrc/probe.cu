// probe.cu -- FMA probes of the GPU, built as libqnsch_probe.so: measurement
// tooling with no counterpart in the paper and no part of the solver's ABI
// (include/qnsch.h).  bench.py runs qnsch_fma_probe in its own process to get
// the FP64 peak it divides the FP64 kernels' achieved rate by: each thread runs
// eight independent FMA chains, so the pipe, not the dependent-instruction
// latency, sets the rate.  qnsch_fp64_issue_probe gives the SM cycles one
// warp-wide FP64 FMA holds a sub-partition for, as a function of the active
// lanes and of the independent chains per lane: the cost model behind the
// solver's launch shapes.
//
// Exported calls (status: 0 ok, -1 invalid argument, -2 no device, -3 out of
// memory, -9 CUDA error; the codes of include/qnsch.h):
//
//   int qnsch_fma_probe(int fp64, int blocks_per_sm, int iters, double* tflops);
//     blocks_per_sm x (SM count) blocks of 256 threads; each thread runs eight
//     independent chains of 16 x iters fused multiply-adds in FP64 (fp64 != 0)
//     or FP32; five launches are timed after three untimed ones with CUDA
//     events on the legacy default stream.  *tflops = 2 x FMAs / s / 1e12.
//     Allocates and frees one scratch array of blocks x 256 elements and
//     synchronises.  blocks_per_sm in [1, 64], iters in [1, 2^24].
//
//   int qnsch_fp64_issue_probe(int warps_per_block, int active_lanes, int chains,
//                              int iters, double* cycles_per_instr);
//     one block of warps_per_block warps per SM; in every warp the lanes below
//     active_lanes run `chains` (1, 2, 4 or 8) independent chains of 16 x iters
//     FP64 FMAs; thread 0 reads the SM cycle counter around the loop.
//     *cycles_per_instr = the slowest block's cycles (best of three launches
//     after one untimed) / FMAs one warp issues / warps sharing one of the
//     SM's four sub-partitions.  warps_per_block and active_lanes in [1, 32],
//     iters in [1, 2^20].
//
//   int qnsch_stage_probe(int mode, int threads, int nb, int K, int stages,
//                         double* us_per_stage);
//     the cost of one dependent stage of a multigrid sweep: `stages` stages in
//     which nb thread blocks of `threads` threads each run a dependent chain
//     of K FP64 FMAs per thread.  mode 0: one cooperative launch of one block
//     per SM, the stages separated by an inter-block barrier (an arrival
//     counter in global memory, every wait bounded by about 2 s of SM clock;
//     blocks >= nb skip the stages); mode 1: one launch per stage, captured
//     into a CUDA graph, each with programmatic stream serialisation (the
//     solver's own launch form).  *us_per_stage = best of five timed runs /
//     stages, in microseconds.  threads in {32, 64, ..., 1024}, nb in
//     [1, SM count], K in [0, 4096], stages in [1, 4096]; a barrier wait that
//     runs out of time gives -6 (QNSCH_ETIMEOUT).
//
//   int qnsch_rcp_check(int n, const double* x, double* y_fast, double* y_ieee);
//     host arrays of n doubles: y_fast = the FP64 reciprocal the block solves
//     use (qrcp of qnsch_dev.cuh: Newton-Raphson from rcp.approx.ftz.f64),
//     y_ieee = 1.0 / x (IEEE division), both computed on the device.
//     n in [1, 2^24]; allocates and frees 3 n doubles; synchronises.
#include <cuda_runtime.h>

#include "qnsch.h"
#include "qnsch_dev.cuh"

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

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// mode 0 of qnsch_stage_probe: the stages in one launch, blocks [0, nb) in
// each, separated by an arrival counter (cumulative target nb per stage)
__global__ void k_stage_persist(unsigned* ctr, int* err, double* sink, int S, int nb, int K) {
  double x = 1.0 + threadIdx.x;
  unsigned target = 0;
  for (int s = 0; s < S; ++s) {
    if ((int)blockIdx.x < nb) {
      if (nb > 1 && s > 0) {
        if (threadIdx.x == 0) {
          const long long t0 = clock64();
          while (ld_acquire_u32(ctr) < target) {
            if (*(volatile int*)err) break;
            if (clock64() - t0 > 4000000000LL) {
              atomicExch(err, 1);
              break;
            }
          }
          __threadfence();
        }
        __syncthreads();
      }
      for (int k = 0; k < K; ++k) x = fma(x, 1.0000001, 1e-9);
      __syncthreads();
      if (nb > 1 && threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
      }
    }
    target += nb;
  }
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x;
}

// mode 1 of qnsch_stage_probe: one stage per launch
__global__ void k_stage_one(double* sink, int K) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  double x = 1.0 + threadIdx.x;
  for (int k = 0; k < K; ++k) x = fma(x, 1.0000001, 1e-9);
  sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = x;
}

int run_stage_probe(int mode, int threads, int nb, int K, int S, double* us) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ENODEV;
  }
  if (nb > sms) return QNSCH_EINVAL;
  unsigned* ctr = nullptr;
  int* err = nullptr;
  double* sink = nullptr;
  if (cudaMalloc(&ctr, sizeof(unsigned)) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&sink, (size_t)sms * threads * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ctr);
    cudaFree(err);
    return QNSCH_ENOMEM;
  }
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraphExec_t ge = nullptr;
  int rc = QNSCH_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    rc = QNSCH_ECUDA;
  if (rc == QNSCH_OK && mode == 1) {  // the graph of S dependent launches
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = QNSCH_ECUDA;
    for (int s = 0; s < S && rc == QNSCH_OK; ++s) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(nb);
      cfg.blockDim = dim3(threads);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if (cudaLaunchKernelEx(&cfg, k_stage_one, sink, K) != cudaSuccess) rc = QNSCH_ECUDA;
    }
    if (rc == QNSCH_OK) {
      if (cudaStreamEndCapture(st, &g) != cudaSuccess || cudaGraphInstantiate(&ge, g, 0) != cudaSuccess)
        rc = QNSCH_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
  }
  float best = 0.f;
  for (int rep = 0; rep < 6 && rc == QNSCH_OK; ++rep) {  // the first run warms up
    if (mode == 0) {
      cudaMemsetAsync(ctr, 0, sizeof(unsigned), st);
      cudaMemsetAsync(err, 0, sizeof(int), st);
    }
    cudaEventRecord(e0, st);
    if (mode == 0) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(sms);
      cfg.blockDim = dim3(threads);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      if (cudaLaunchKernelEx(&cfg, k_stage_persist, ctr, err, sink, S, nb, K) != cudaSuccess)
        rc = QNSCH_ECUDA;
    } else if (cudaGraphLaunch(ge, st) != cudaSuccess) {
      rc = QNSCH_ECUDA;
    }
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (rc == QNSCH_OK && (cudaStreamSynchronize(st) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = QNSCH_ECUDA;
    if (rc == QNSCH_OK && mode == 0) {
      int herr = 0;
      if (cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = QNSCH_ECUDA;
      else if (herr) rc = QNSCH_ETIMEOUT;
    }
    if (rc == QNSCH_OK && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (rc == QNSCH_OK) *us = 1e3 * (double)best / S;
  if (rc != QNSCH_OK) cudaGetLastError();
  if (ge) cudaGraphExecDestroy(ge);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(ctr);
  cudaFree(err);
  cudaFree(sink);
  return rc;
}

__global__ void k_rcp_check(const double* x, double* yf, double* yi, int n) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  yf[t] = qn::qrcp(x[t]);
  yi[t] = 1.0 / x[t];
}

}  // namespace

extern "C" int qnsch_rcp_check(int n, const double* x, double* y_fast, double* y_ieee) {
  if (n < 1 || n > (1 << 24) || !x || !y_fast || !y_ieee) return QNSCH_EINVAL;
  int nd = 0;
  if (cudaGetDeviceCount(&nd) != cudaSuccess || nd == 0) {
    cudaGetLastError();
    return QNSCH_ENODEV;
  }
  double* d = nullptr;
  const size_t bytes = (size_t)n * sizeof(double);
  if (cudaMalloc(&d, 3 * bytes) != cudaSuccess) {
    cudaGetLastError();
    return QNSCH_ENOMEM;
  }
  int rc = QNSCH_OK;
  if (cudaMemcpy(d, x, bytes, cudaMemcpyHostToDevice) != cudaSuccess) rc = QNSCH_ECUDA;
  if (rc == QNSCH_OK) {
    k_rcp_check<<<(n + 255) / 256, 256>>>(d, d + n, d + 2 * (size_t)n, n);
    if (cudaMemcpy(y_fast, d + n, bytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(y_ieee, d + 2 * (size_t)n, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = QNSCH_ECUDA;
  }
  if (rc != QNSCH_OK) cudaGetLastError();
  cudaFree(d);
  return rc;
}

extern "C" int qnsch_stage_probe(int mode, int threads, int nb, int K, int stages,
                                 double* us_per_stage) {
  if (!us_per_stage || (mode != 0 && mode != 1) || threads < 32 || threads > 1024 ||
      threads % 32 || nb < 1 || K < 0 || K > 4096 || stages < 1 || stages > 4096)
    return QNSCH_EINVAL;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
    cudaGetLastError();
    return QNSCH_ENODEV;
  }
  return run_stage_probe(mode, threads, nb, K, stages, us_per_stage);
}

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
