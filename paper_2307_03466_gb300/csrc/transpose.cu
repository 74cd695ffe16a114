// Stable transpose of a CSR matrix on the device, for the set-up of an LP handle:
// column j of A^T lists the rows of column j of A in ascending order, with their
// values.  The nonzeros, already in row-major order, are sorted by column index with
// a least-significant-digit radix sort (8 bits per pass, as many passes as the
// column count needs), which is stable within and across blocks; the sorted order
// then gives each entry's row and value.  Every step is deterministic: the only
// atomics are integer counts.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace scylla {

namespace {

constexpr int kTpThreads = 256;
constexpr int kTpItems = 16;
constexpr int kTpChunk = kTpThreads * kTpItems;  // keys per block and pass
constexpr int kScanThreads = 1024;

// row index of every nonzero: a thread per row fills its entries
__global__ void k_tp_rowof(int m, const int* __restrict__ rowptr, int* __restrict__ rowof) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int p1 = rowptr[i + 1];
    for (int p = rowptr[i]; p < p1; ++p) rowof[p] = i;
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

// Exclusive prefix sum of data[0, len) in place, data[len] = the total (integer
// sums, so the grouping does not matter): block b owns the segment [b seg,
// (b + 1) seg); pass 1 sums each segment, pass 2 scans the segment sums in one
// block, pass 3 rescans each segment from its offset in chunks of
// kScanThreads * kScanItems (each thread a run of kScanItems, then a block scan of
// the run totals).
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;
constexpr int kScanMaxBlocks = 1024;

// exclusive block-wide scan of one value per thread (kScanThreads threads);
// returns the thread's offset and the block total in *total
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* sh, long long* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  long long x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    long long z = lane < kScanThreads / 32 ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    if (lane < kScanThreads / 32) sh[32 + lane] = z;  // inclusive over warps
  }
  __syncthreads();
  const long long before = w > 0 ? sh[32 + w - 1] : 0;
  *total = sh[32 + kScanThreads / 32 - 1];
  __syncthreads();  // sh is reused by the next call
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int* __restrict__ data, long long len,
                                                              long long seg, long long* __restrict__ bsum) {
  __shared__ long long sh[64];
  const long long b0 = blockIdx.x * seg, b1 = b0 + seg < len ? b0 + seg : len;
  long long s = 0;
  for (long long i = b0 + threadIdx.x; i < b1; i += kScanThreads) s += data[i];
  long long total = 0;
  block_exclusive_scan(s, sh, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(long long* __restrict__ bsum, int nb,
                                                           int* __restrict__ data, long long len) {
  __shared__ long long sh[64];
  const long long v = int(threadIdx.x) < nb ? bsum[threadIdx.x] : 0;
  long long total = 0;
  const long long ex = block_exclusive_scan(v, sh, &total);
  if (int(threadIdx.x) < nb) bsum[threadIdx.x] = ex;
  if (threadIdx.x == 0) data[len] = int(total);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(int* __restrict__ data, long long len, long long seg,
                                                            const long long* __restrict__ bsum) {
  __shared__ long long sh[64];
  const long long b0 = blockIdx.x * seg, b1 = b0 + seg < len ? b0 + seg : len;
  long long carry = bsum[blockIdx.x];
  for (long long c0 = b0; c0 < b1; c0 += kScanChunk) {
    const long long t0 = c0 + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      v[k] = t0 + k < b1 ? data[t0 + k] : 0;
      s += v[k];
    }
    long long total = 0;
    long long run = carry + block_exclusive_scan(s, sh, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
      if (t0 + k < b1) {
        data[t0 + k] = int(run);
        run += v[k];
      }
    carry += total;
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

// the scan of data[0, len) with data[len] = total; bsum holds kScanMaxBlocks entries
void scan_exclusive(int* data, long long len, long long* bsum, cudaStream_t st) {
  long long nb = (len + kScanChunk - 1) / kScanChunk;
  if (nb > kScanMaxBlocks) nb = kScanMaxBlocks;
  if (nb < 1) nb = 1;
  long long seg = (len + nb - 1) / nb;
  seg = (seg + kScanChunk - 1) / kScanChunk * kScanChunk;
  nb = len > 0 ? (len + seg - 1) / seg : 1;
  k_scan_reduce<<<int(nb), kScanThreads, 0, st>>>(data, len, seg, bsum);
  k_scan_top<<<1, kScanThreads, 0, st>>>(bsum, int(nb), data, len);
  k_scan_down<<<int(nb), kScanThreads, 0, st>>>(data, len, seg, bsum);
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
  return ints * sizeof(int) + 8 * sizeof(long long) * kScanMaxBlocks;
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
  // the scan's segment sums after the histogram (8-byte aligned)
  const size_t hist_ints = size_t(256 * ((nnz + kTpChunk - 1) / kTpChunk)) + 1;
  long long* bsum = reinterpret_cast<long long*>(
      (reinterpret_cast<uintptr_t>(hist + hist_ints) + 15) & ~uintptr_t(15));
  const long long nb = (nnz + kTpChunk - 1) / kTpChunk;
  // column counts -> column pointers
  k_tp_count<<<grid_for(nnz), 256, 0, st>>>(nnz, cols, colptr);
  scan_exclusive(colptr, n, bsum, st);
  k_tp_rowof<<<grid_for(m), 256, 0, st>>>(m, rowptr, rowof);
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
    scan_exclusive(hist, 256 * nb, bsum, st);
    k_tp_scatter<<<int(nb), kTpThreads, 0, st>>>(kin, iin, kout, iout, nnz, shift, hist);
    kin = kout;
    iin = iout;
  }
  k_tp_gather<<<grid_for(nnz), 256, 0, st>>>(nnz, iin, rowof, vals, rows_out, vals_out);
  return cudaGetLastError();
}

}  // namespace scylla
