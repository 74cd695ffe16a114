// Stable transpose of a CSR matrix on the device, for the set-up of an LP handle:
// column j of A^T lists the rows of column j of A in ascending order, with their
// values.  The nonzeros, already in row-major order, are sorted by column index with
// a least-significant-digit radix sort (8 bits per pass, as many passes as the
// column count needs), which is stable within and across blocks; the sorted order
// then gives each entry's row and value.  Every step is deterministic: the only
// atomics are integer counts.
#include <cuda_runtime.h>

#include "internal.h"

namespace scylla {

namespace {

constexpr int kTpThreads = 256;
constexpr int kTpItems = 16;
constexpr int kTpChunk = kTpThreads * kTpItems;  // keys per block and pass
constexpr int kScanThreads = 1024;

// row index of every nonzero (binary search in the row pointers: long rows cost the
// same as short ones)
__global__ void k_tp_rowof(int m, long long nnz, const int* __restrict__ rowptr, int* __restrict__ rowof) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x) {
    int lo = 0, hi = m;  // the row i with rowptr[i] <= p < rowptr[i + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (rowptr[mid] <= p) lo = mid;
      else hi = mid;
    }
    rowof[p] = lo;
  }
}

// entries per column
__global__ void k_tp_count(long long nnz, const int* __restrict__ cols, int* __restrict__ count) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz; p += (long long)gridDim.x * blockDim.x)
    atomicAdd(count + cols[p], 1);
}

// digit histogram of each block's chunk, stored digit-major: hist[d * nblocks + b]
__global__ void __launch_bounds__(kTpThreads) k_tp_hist(const int* __restrict__ keys, long long nnz, int shift,
                                                        int* __restrict__ hist) {
  __shared__ int cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kTpChunk;
  for (int r = 0; r < kTpItems; ++r) {
    const long long p = base + r * kTpThreads + threadIdx.x;
    if (p < nnz) atomicAdd(&cnt[(keys[p] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[threadIdx.x * gridDim.x + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive prefix sum of data[0, len) in place, one block: each thread scans a
// contiguous segment; data[len] receives the total
__global__ void __launch_bounds__(kScanThreads) k_tp_scan(int* __restrict__ data, long long len) {
  __shared__ long long part[kScanThreads];
  const long long seg = (len + kScanThreads - 1) / kScanThreads;
  const long long b = threadIdx.x * seg, e = b + seg < len ? b + seg : len;
  long long s = 0;
  for (long long i = b; i < e; ++i) s += data[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long run = 0;
    for (int t = 0; t < kScanThreads; ++t) {
      const long long v = part[t];
      part[t] = run;
      run += v;
    }
    data[len] = int(run);
  }
  __syncthreads();
  long long run = part[threadIdx.x];
  for (long long i = b; i < e; ++i) {
    const int v = data[i];
    data[i] = int(run);
    run += v;
  }
}

// one stable pass: every key of the block's chunk goes to
// offset[digit][block] + (keys of that digit earlier in the chunk).  The chunk is read
// in rounds of 256 keys; within a round a key's rank is the number of same-digit keys
// in lower lanes of its warp plus those of lower warps and of earlier rounds.
__global__ void __launch_bounds__(kTpThreads) k_tp_scatter(const int* __restrict__ keys_in, const int* __restrict__ idx_in,
                                                           int* __restrict__ keys_out, int* __restrict__ idx_out,
                                                           long long nnz, int shift, const int* __restrict__ offsets) {
  __shared__ int base[256];
  __shared__ int wcnt[kTpThreads / 32][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  base[threadIdx.x] = offsets[threadIdx.x * gridDim.x + blockIdx.x];
  const long long chunk = (long long)blockIdx.x * kTpChunk;
  for (int r = 0; r < kTpItems; ++r) {
#pragma unroll
    for (int v = 0; v < kTpThreads / 32; ++v) wcnt[v][threadIdx.x] = 0;
    __syncthreads();
    const long long p = chunk + r * kTpThreads + threadIdx.x;
    const bool valid = p < nnz;
    const int key = valid ? keys_in[p] : 0;
    const int d = valid ? (key >> shift) & 255 : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    int run = base[threadIdx.x];
#pragma unroll
    for (int v = 0; v < kTpThreads / 32; ++v) {
      const int c = wcnt[v][threadIdx.x];
      wcnt[v][threadIdx.x] = run;
      run += c;
    }
    base[threadIdx.x] = run;
    __syncthreads();
    if (valid) {
      const int dest = wcnt[w][d] + rank;
      keys_out[dest] = key;
      idx_out[dest] = idx_in ? idx_in[p] : int(p);
    }
    __syncthreads();
  }
}

__global__ void k_tp_gather(long long nnz, const int* __restrict__ order, const int* __restrict__ rowof,
                            const double* __restrict__ vals, int* __restrict__ rows_out, double* __restrict__ vals_out) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x) {
    const int p = order[q];
    rows_out[q] = rowof[p];
    vals_out[q] = vals[p];
  }
}

int grid_for(long long work) {
  const long long g = (work + 255) / 256;
  const long long cap = 8LL * device_sm_count();
  return int(g < 1 ? 1 : (g < cap ? g : cap));
}

}  // namespace

size_t transpose_scratch_bytes(int n, long long nnz) {
  const long long nb = (nnz + kTpChunk - 1) / kTpChunk;
  const size_t ints = size_t(5 * nnz) + size_t(256 * (nb > 0 ? nb : 1) + 1) + size_t(n) + 1 + 64;
  return ints * sizeof(int);
}

cudaError_t transpose_device(int m, int n, long long nnz, const int* rowptr, const int* cols, const double* vals,
                             int* colptr, int* rows_out, double* vals_out, void* scratch, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(colptr, 0, sizeof(int) * (size_t(n) + 1), st);
  if (e != cudaSuccess || nnz == 0) return e;
  int* keys[2];
  int* idx[2];
  int* s = static_cast<int*>(scratch);
  keys[0] = s;
  keys[1] = s + nnz;
  idx[0] = s + 2 * nnz;
  idx[1] = s + 3 * nnz;
  int* rowof = s + 4 * nnz;
  int* hist = s + 5 * nnz;
  const long long nb = (nnz + kTpChunk - 1) / kTpChunk;
  // column counts -> column pointers
  k_tp_count<<<grid_for(nnz), 256, 0, st>>>(nnz, cols, colptr);
  k_tp_scan<<<1, kScanThreads, 0, st>>>(colptr, n);
  k_tp_rowof<<<grid_for(nnz), 256, 0, st>>>(m, nnz, rowptr, rowof);
  // radix passes over the column bits
  int bits = 0;
  while (bits < 31 && (1LL << bits) < n) ++bits;
  const int passes = bits == 0 ? 1 : (bits + 7) / 8;
  const int* kin = cols;
  const int* iin = nullptr;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = 8 * pass;
    int* kout = keys[pass & 1];
    int* iout = idx[pass & 1];
    k_tp_hist<<<int(nb), kTpThreads, 0, st>>>(kin, nnz, shift, hist);
    k_tp_scan<<<1, kScanThreads, 0, st>>>(hist, 256 * nb);
    k_tp_scatter<<<int(nb), kTpThreads, 0, st>>>(kin, iin, kout, iout, nnz, shift, hist);
    kin = kout;
    iin = iout;
  }
  k_tp_gather<<<grid_for(nnz), 256, 0, st>>>(nnz, iin, rowof, vals, rows_out, vals_out);
  return cudaGetLastError();
}

}  // namespace scylla
