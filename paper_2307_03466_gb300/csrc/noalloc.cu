// Primal residual of a caller-owned LP without any device allocation.
//
// Some callers cannot allocate device memory at all: plugins that their host
// application hands a fixed memory pool, real-time loops that forbid allocator calls
// (cudaMalloc and cudaFree can block and synchronise the device), and processes that
// share a GPU under a fixed memory budget set elsewhere.  For them,
// scylla_primal_residual_noalloc evaluates the relative primal residual
// eps_p = ||A x - proj_[lo,hi](A x)||_2 / (1 + ||b||_2) of a point x on an LP the
// caller keeps in its own device memory.  The per-block partial sums that the
// residual kernel of the solver keeps in its handle's scratch live here in one
// file-scope __device__ array instead, so the call allocates nothing.
//
// That array is shared by every call on a device and keeps the last call's
// contents; calls that overlap on the GPU (on different streams, or from different
// host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "internal.h"

namespace {

constexpr int kNaThreads = 256;       // one row per thread
constexpr int kNaMaxBlocks = 8192;    // so at most 2,097,152 rows per call
constexpr int kNaSums = 2;            // ||r_p||^2 and ||b||^2

struct NoAllocScratch {
  double partial[kNaMaxBlocks * kNaSums];
  unsigned int blocks_done;
};

// 128 KiB + 4 bytes per device, held by every GPU that loads the library until exit
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// thread per row: (A x)_i in CSR order, its distance to [lo_i, hi_i] and the row's
// bound magnitude; the last block to finish reduces the per-block sums in a fixed
// order, writes out[0] = ||r_p||_2 and out[1] = eps_p, and clears the counter.
__global__ void __launch_bounds__(kNaThreads) k_primal_residual_noalloc(
    NoAllocScratch* sc, long long m, const long long* __restrict__ rowptr, const int* __restrict__ cols,
    const double* __restrict__ vals, const double* __restrict__ x, const double* __restrict__ lo,
    const double* __restrict__ hi, double* __restrict__ out) {
  const double inf = __longlong_as_double(0x7ff0000000000000ULL);
  double s[kNaSums] = {0.0, 0.0};
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    double ax = 0.0;
    for (long long p = rowptr[i]; p < rowptr[i + 1]; ++p) ax += vals[p] * x[cols[p]];
    const double l = lo[i], h = hi[i];
    const double proj = ax < l ? l : (ax > h ? h : ax);
    const double r = ax - proj;
    s[0] = r * r;
    const double bl = l > -inf ? fabs(l) : 0.0, bh = h < inf ? fabs(h) : 0.0;
    const double b = bl > bh ? bl : bh;
    s[1] = b * b;
  }
  __shared__ double sh[kNaThreads / 32][kNaSums];
  __shared__ int last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kNaSums; ++k) {
    const double t = na_warp_sum(s[k]);
    if (lane == 0) sh[w][k] = t;
  }
  __syncthreads();
  if (threadIdx.x < kNaSums) {
    double t = 0.0;
    for (int q = 0; q < kNaThreads / 32; ++q) t += sh[q][threadIdx.x];
    sc->partial[blockIdx.x * kNaSums + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&sc->blocks_done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t[kNaSums] = {0.0, 0.0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < kNaSums; ++k) t[k] += __ldcg(&sc->partial[b * kNaSums + k]);
#pragma unroll
  for (int k = 0; k < kNaSums; ++k) {
    const double v = na_warp_sum(t[k]);
    if (lane == 0) sh[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double rr = 0.0, bb = 0.0;
    for (int q = 0; q < kNaThreads / 32; ++q) {
      rr += sh[q][0];
      bb += sh[q][1];
    }
    const double rn = sqrt(rr);
    out[0] = rn;
    out[1] = rn / (1.0 + sqrt(bb));
    sc->blocks_done = 0u;  // the next call starts from zero
  }
}

// Device address of the scratch array, looked up by the first call on each device
// and kept for the life of the process.  In host code the name g_noalloc_scratch is
// only a host-side stand-in, so a kernel must be given the address that
// cudaGetSymbolAddress returns while that device is current.  After a
// cudaDeviceReset the module is loaded again and the kept address is stale: the
// entry point is not for use across a device reset.
constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
NoAllocScratch* g_na_ptr[kMaxDevices] = {};

int scratch_for_current_device(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    scylla::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return SCYLLA_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    scylla::set_error("device ordinal beyond the supported range");
    return SCYLLA_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> g(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      scylla::set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return SCYLLA_ERR_CUDA;
    }
    g_na_ptr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_na_ptr[dev];
  return SCYLLA_OK;
}

}  // namespace

extern "C" int scylla_primal_residual_noalloc(int64_t m, const int64_t* rowptr, const int32_t* cols,
                                              const double* vals, const double* x, const double* row_lo,
                                              const double* row_hi, double* out, void* cuda_stream) {
  const int64_t max_rows = int64_t(kNaMaxBlocks) * kNaThreads;
  if (m < 1 || m > max_rows) {
    scylla::set_error("scylla_primal_residual_noalloc: need 1 <= m <= " + std::to_string(max_rows) +
                      " rows (its fixed scratch holds " + std::to_string(kNaMaxBlocks) + " block sums), got " +
                      std::to_string(m));
    return SCYLLA_ERR_INVALID_ARG;
  }
  if (!rowptr || !cols || !vals || !x || !row_lo || !row_hi || !out) {
    scylla::set_error("scylla_primal_residual_noalloc: null pointer");
    return SCYLLA_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NoAllocScratch* sc = nullptr;
  const int rc = scratch_for_current_device(&sc);
  if (rc != SCYLLA_OK) return rc;
  // every call clears the arrival counter on its own stream before its kernel: a
  // finished kernel leaves it at zero, but one that failed part way (or a launch
  // that was cancelled) would leave a count that the next call must not inherit
  cudaError_t e = cudaMemsetAsync(&sc->blocks_done, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) {
    scylla::set_error(std::string("scylla_primal_residual_noalloc: clearing the scratch counter: ") +
                      cudaGetErrorString(e));
    return SCYLLA_ERR_CUDA;
  }
  const int blocks = int((m + kNaThreads - 1) / kNaThreads);
  k_primal_residual_noalloc<<<blocks, kNaThreads, 0, st>>>(sc, (long long)m, (const long long*)rowptr, cols, vals,
                                                            x, row_lo, row_hi, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    scylla::set_error(std::string("scylla_primal_residual_noalloc launch: ") + cudaGetErrorString(e));
    return SCYLLA_ERR_CUDA;
  }
  return SCYLLA_OK;
}
