// noalloc.cu -- mass reduction that allocates no memory (qnsch_mass_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a result:
// code that runs inside a memory-pool or allocator callback (an allocation
// there would re-enter the allocator), host programs whose device memory is
// fully reserved up front by another framework (a caching allocator that holds
// all of HBM), and latency-critical loops that must not call cudaMalloc,
// which can synchronise the device.  The handle-based qnsch_mass needs a
// solver handle, which allocates the whole multigrid hierarchy.  This entry
// point instead takes the caller's concentration array and output pointer and
// keeps its only scratch (one partial sum pair per thread block) in a fixed,
// file-scope device array.
#include <cuda_runtime.h>

#include <mutex>

#include "qnsch.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_BLOCK = NA_THREADS * 8;  // each thread sums 8 cells
constexpr int NA_MAX_BLOCKS = QNSCH_NOALLOC_MAX_CELLS / NA_CELLS_PER_BLOCK;

// Block partials [NA_MAX_BLOCKS][2]: 64 KiB, held by every GPU that loads the
// library until the process exits.  Every block writes its own pair before the
// finishing kernel reads it, so nothing has to start at zero.
static __device__ __align__(256) double g_mass_partials[NA_MAX_BLOCKS * 2];

constexpr int NA_MAX_DEVICES = 64;
void* g_partials_addr[NA_MAX_DEVICES] = {};
std::mutex g_setup_mu;

// Device address of g_mass_partials for the current device (the host-side
// symbol is only a stand-in and must never be passed to a kernel).  The
// address is looked up once per device ordinal and kept for the life of the
// process; a device reset (cudaDeviceReset) unloads the module and leaves it
// stale, so a program that resets a device must not call this entry point
// again in the same process.
int partials_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return QNSCH_ENODEV;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_mass_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return QNSCH_ECUDA;
    }
    g_partials_addr[dev] = p;
  }
  *out = g_partials_addr[dev];
  return QNSCH_OK;
}

// rho(c) = 1 / (ia c + ib) with ia = (rho2 - rho1)/(rho1 rho2), ib = 1/rho2 (Sec. 2.1)
__global__ void k_mass_partials(const double* __restrict__ c, long long n, double ia, double ib,
                                double* __restrict__ part) {
  __shared__ double sr[NA_THREADS / 32], src[NA_THREADS / 32];
  long long base = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int q = 0; q < NA_CELLS_PER_BLOCK / NA_THREADS; ++q) {
    long long k = base + (long long)q * NA_THREADS + threadIdx.x;
    if (k < n) {
      double cc = c[k];
      double r = 1.0 / (ia * cc + ib);
      a += r;
      b += r * cc;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    sr[warp] = a;
    src[warp] = b;
  }
  __syncthreads();
  if (warp == 0) {
    a = lane < NA_THREADS / 32 ? sr[lane] : 0.0;
    b = lane < NA_THREADS / 32 ? src[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      part[2 * blockIdx.x] = a;
      part[2 * blockIdx.x + 1] = b;
    }
  }
}

// one block: fixed-order sum of the partials, scaled by h^2
__global__ void k_mass_finish(const double* __restrict__ part, int nblocks, double h2,
                              double* __restrict__ out2) {
  __shared__ double sa[NA_THREADS], sb[NA_THREADS];
  double a = 0.0, b = 0.0;
  for (int p = threadIdx.x; p < nblocks; p += NA_THREADS) {
    a += part[2 * p];
    b += part[2 * p + 1];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out2[0] = h2 * sa[0];
    out2[1] = h2 * sb[0];
  }
}

}  // namespace

extern "C" int qnsch_mass_noalloc(const double* c, int m1, int m2, double h, double rho1,
                                  double rho2, double* out2, void* stream) {
  if (!c || !out2 || m1 < 1 || m2 < 1 || !(h > 0) || !(rho1 > 0) || !(rho2 > 0))
    return QNSCH_EINVAL;
  long long n = (long long)m1 * (long long)m2;
  if (n > QNSCH_NOALLOC_MAX_CELLS) return QNSCH_EINVAL;
  void* part = nullptr;
  int rc = partials_address(&part);
  if (rc) return rc;
  int nblocks = (int)((n + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
  cudaStream_t s = (cudaStream_t)stream;
  double ia = (rho2 - rho1) / (rho1 * rho2), ib = 1.0 / rho2;
  k_mass_partials<<<nblocks, NA_THREADS, 0, s>>>(c, n, ia, ib, (double*)part);
  k_mass_finish<<<1, NA_THREADS, 0, s>>>((const double*)part, nblocks, h * h, out2);
  return cudaGetLastError() == cudaSuccess ? QNSCH_OK : QNSCH_ECUDA;
}
