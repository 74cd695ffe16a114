// Set-up kernels of an LP handle (run once per create): the diagonal
// preconditioning of Section 2.1 (PDLP's Ruiz iterations, then one Pock-Chambolle
// step), the scaled copies of the matrix values, fills, the column kinds of the
// pump's objective update (Section 2.4), and the norms behind the initial step size
// and primal weight.
//
// The preconditioning and scaling kernels walk the same warp tiles as the SpMV
// (contiguous rows with at most kTileNnz nonzeros and kTileRows rows, or one long
// row): the rows of a tile are spread over the warp, L = 32 / rows (a power of two)
// lanes per row, so a long row is read by the whole warp and short rows by one lane
// each.  A row's L partial results are combined by a shuffle tree.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

namespace scylla {

namespace {

constexpr int kSetupThreads = 256;

// lanes per row of a tile of nr rows: the largest power of two L with L * nr <= 32
__device__ __forceinline__ int setup_row_lanes(int nr) {
  if (nr >= 32) return 1;
  const int l = 32 / (nr > 0 ? nr : 1);
  return 1 << (31 - __clz(l));
}

int setup_grid(long long warps_or_items, int per_block) {
  long long g = (warps_or_items + per_block - 1) / per_block;
  const long long cap = 8LL * device_sm_count();
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return int(g);
}

__global__ void k_fill_f64(double* __restrict__ p, long long count, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

// new column bounds in the scaled space, with the rounding of the scaled vectors at
// create: l~_j = l_j / C_j, u~_j = u_j / C_j
__global__ void k_scale_col_bounds(long long n, const double* __restrict__ l, const double* __restrict__ u,
                                   const double* __restrict__ C, double* __restrict__ l64, double* __restrict__ u64,
                                   float* __restrict__ l32, float* __restrict__ u32) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const double cj = C[j], lj = l[j] / cj, uj = u[j] / cj;
    l64[j] = lj;
    u64[j] = uj;
    if (l32) {
      l32[j] = float(lj);
      u32[j] = float(uj);
    }
  }
}

// new row bounds in the scaled space, with the rounding of the scaled vectors at
// create: lo~_i = lo_i R_i, hi~_i = hi_i R_i
__global__ void k_scale_row_bounds(long long m, const double* __restrict__ lo, const double* __restrict__ hi,
                                   const double* __restrict__ R, double* __restrict__ lo64,
                                   double* __restrict__ hi64, float* __restrict__ lo32, float* __restrict__ hi32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const double ri = R[i], a = lo[i] * ri, b = hi[i] * ri;
    lo64[i] = a;
    hi64[i] = b;
    if (lo32) {
      lo32[i] = float(a);
      hi32[i] = float(b);
    }
  }
}

// Hessian diagonal in the scaled space: q~_j = (q_j C_j) C_j
__global__ void k_scale_hessian(long long n, const double* __restrict__ q, const double* __restrict__ C,
                                double* __restrict__ q64, float* __restrict__ q32) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const double cj = C[j], v = (q[j] * cj) * cj;
    q64[j] = v;
    if (q32) q32[j] = float(v);
  }
}

// a new objective in the scaled space: c~_j = c_j C_j, q~_j = (q_j C_j) C_j
__global__ void k_scale_objective(long long n, const double* __restrict__ c, const double* __restrict__ q,
                                  const double* __restrict__ C, double* __restrict__ c64, float* __restrict__ c32,
                                  double* __restrict__ q64, float* __restrict__ q32) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const double cj = C[j], a = c[j] * cj, b = (q[j] * cj) * cj;
    c64[j] = a;
    q64[j] = b;
    if (c32) c32[j] = float(a);
    if (q32) q32[j] = float(b);
  }
}

// kind_j = 1 for an integer column, 0 otherwise; aux_j = -1 (no auxiliary columns)
__global__ void k_column_kinds(long long n, const uint8_t* __restrict__ is_int, int* __restrict__ kind,
                               int* __restrict__ aux_of) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    kind[j] = is_int[j] ? 1 : 0;
    aux_of[j] = -1;
  }
}

// One preconditioning factor per row of one side of A (kRow: the rows of A, self =
// R, other = C; else the rows of A^T, self = C, other = R):
//   out_i = self_i / sqrt(red_j |a~_ij|),  a~_ij = (self_i |a_ij|) other_j on rows and
//   (other_i |a_ij|) self_j on columns (the product order of the scaled values),
// red = max for a Ruiz iteration and sum for the Pock-Chambolle step (alpha = 1);
// a row without nonzeros keeps its factor.  The warp takes tiles t = first,
// first + step, ...
template <bool kMax, bool kRow>
__device__ __forceinline__ void side_factor(int first, int step, const int2* __restrict__ tiles, int ntiles,
                                            const int* __restrict__ ptr, const int* __restrict__ idx,
                                            const double* __restrict__ vals, const double* __restrict__ self,
                                            const double* __restrict__ other, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int t = first; t < ntiles; t += step) {
    const int r0 = tiles[t].x, nr = tiles[t + 1].x - r0;
    const int L = setup_row_lanes(nr), rl = lane / L, sub = lane - rl * L;
    const bool mine = rl < nr;
    const int row = r0 + rl;
    double acc = 0.0, si = 0.0;
    if (mine) {
      si = self[row];
      const int q1 = ptr[row + 1];
      for (int p = ptr[row] + sub; p < q1; p += L) {
        const double a = fabs(vals[p]), o = other[idx[p]];
        const double term = kRow ? (si * a) * o : (o * a) * si;
        acc = kMax ? fmax(acc, term) : acc + term;
      }
    }
    for (int off = L >> 1; off > 0; off >>= 1) {
      const double v = __shfl_down_sync(0xffffffffu, acc, off);
      acc = kMax ? fmax(acc, v) : acc + v;
    }
    if (mine && sub == 0) out[row] = acc > 0.0 ? si / sqrt(acc) : si;
  }
}

// both sides of one preconditioning pass in one launch (each reads the pass's R and
// C and writes R2 and C2): blocks [0, gr) take the rows of A, the rest those of A^T
template <bool kMax>
__global__ void __launch_bounds__(kSetupThreads) k_side_factors(DevSetup s, int gr, const double* __restrict__ r,
                                                               const double* __restrict__ c, double* __restrict__ r2,
                                                               double* __restrict__ c2) {
  const int wpb = kSetupThreads / 32, w = int(threadIdx.x >> 5);
  if (int(blockIdx.x) < gr) {
    side_factor<kMax, true>(int(blockIdx.x) * wpb + w, gr * wpb, s.a_tiles, s.a_ntiles, s.a_rowptr, s.a_cols,
                            s.a_vals64, r, c, r2);
  } else {
    const int b = int(blockIdx.x) - gr, gc = int(gridDim.x) - gr;
    side_factor<kMax, false>(b * wpb + w, gc * wpb, s.t_tiles, s.t_ntiles, s.t_rowptr, s.t_cols, s.t_vals64, c,
                             r, c2);
  }
}

// a~_ij = (a_ij R_i) C_j in place on one side (kRow: A, self = R; else A^T, self =
// C), with the FP32 shadow when vals32 is given; both sides round the same product.
template <bool kRow>
__global__ void __launch_bounds__(kSetupThreads)
    k_scale_side(const int2* __restrict__ tiles, int ntiles, const int* __restrict__ ptr, const int* __restrict__ idx,
                 double* __restrict__ vals, float* __restrict__ vals32, const double* __restrict__ self,
                 const double* __restrict__ other) {
  const int lane = threadIdx.x & 31;
  const int warp = int((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = int((gridDim.x * blockDim.x) >> 5);
  for (int t = warp; t < ntiles; t += nwarps) {
    const int r0 = tiles[t].x, nr = tiles[t + 1].x - r0;
    const int L = setup_row_lanes(nr), rl = lane / L, sub = lane - rl * L;
    if (rl >= nr) continue;
    const int row = r0 + rl;
    const double si = self[row];
    const int q1 = ptr[row + 1];
    for (int p = ptr[row] + sub; p < q1; p += L) {
      const double o = other[idx[p]];
      const double v = kRow ? (vals[p] * si) * o : (vals[p] * o) * si;
      vals[p] = v;
      if (vals32) vals32[p] = float(v);
    }
  }
}

// part[4 b + (0, 1, 2, 3)] = (max |a~|, sum a~^2, sum c~^2, sum q~^2) over block b's
// grid-stride slices, q~_i = max(|lo~_i|, |hi~_i|) over the finite bounds of row i;
// each block sums its threads' partials in thread order.
__global__ void __launch_bounds__(kSetupThreads)
    k_setup_norms(const double* __restrict__ a, long long nnz, const double* __restrict__ c, long long n,
                  const double* __restrict__ lo, const double* __restrict__ hi, long long m,
                  double* __restrict__ part) {
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, stride = (long long)gridDim.x * blockDim.x;
  double mx = 0.0, s = 0.0, cs = 0.0, qs = 0.0;
  for (long long p = t0; p < nnz; p += stride) {
    const double v = a[p];
    mx = fmax(mx, fabs(v));
    s += v * v;
  }
  for (long long j = t0; j < n; j += stride) cs += c[j] * c[j];
  for (long long i = t0; i < m; i += stride) {
    const double x = isfinite(lo[i]) ? fabs(lo[i]) : 0.0, y = isfinite(hi[i]) ? fabs(hi[i]) : 0.0;
    const double q = fmax(x, y);
    qs += q * q;
  }
  __shared__ double sh[4][kSetupThreads];
  sh[0][threadIdx.x] = mx;
  sh[1][threadIdx.x] = s;
  sh[2][threadIdx.x] = cs;
  sh[3][threadIdx.x] = qs;
  __syncthreads();
  if (threadIdx.x < 4) {
    const int k = int(threadIdx.x);
    double r = 0.0;
    for (int q = 0; q < int(blockDim.x); ++q) r = k == 0 ? fmax(r, sh[0][q]) : r + sh[k][q];
    part[4 * blockIdx.x + k] = r;
  }
}

template <bool kMax>
void side_factors(const DevSetup& s, double* r, double* c, double* r2, double* c2, cudaStream_t st) {
  const int gr = setup_grid(s.a_ntiles, kSetupThreads / 32), gc = setup_grid(s.t_ntiles, kSetupThreads / 32);
  k_side_factors<kMax><<<gr + gc, kSetupThreads, 0, st>>>(s, gr, r, c, r2, c2);
}

}  // namespace

cudaError_t fill_f64(double* p, long long count, double v, cudaStream_t st) {
  if (count > 0) k_fill_f64<<<setup_grid(count, kSetupThreads), kSetupThreads, 0, st>>>(p, count, v);
  return cudaGetLastError();
}

cudaError_t scale_col_bounds(long long n, const double* l, const double* u, const double* C, double* l64,
                             double* u64, float* l32, float* u32, cudaStream_t st) {
  if (n > 0)
    k_scale_col_bounds<<<setup_grid(n, kSetupThreads), kSetupThreads, 0, st>>>(n, l, u, C, l64, u64, l32, u32);
  return cudaGetLastError();
}

cudaError_t scale_row_bounds(long long m, const double* lo, const double* hi, const double* R, double* lo64,
                             double* hi64, float* lo32, float* hi32, cudaStream_t st) {
  if (m > 0)
    k_scale_row_bounds<<<setup_grid(m, kSetupThreads), kSetupThreads, 0, st>>>(m, lo, hi, R, lo64, hi64, lo32, hi32);
  return cudaGetLastError();
}

cudaError_t scale_objective(long long n, const double* c, const double* q, const double* C, double* c64,
                            float* c32, double* q64, float* q32, cudaStream_t st) {
  if (n > 0) k_scale_objective<<<setup_grid(n, kSetupThreads), kSetupThreads, 0, st>>>(n, c, q, C, c64, c32, q64, q32);
  return cudaGetLastError();
}

cudaError_t scale_hessian(long long n, const double* q, const double* C, double* q64, float* q32, cudaStream_t st) {
  if (n > 0) k_scale_hessian<<<setup_grid(n, kSetupThreads), kSetupThreads, 0, st>>>(n, q, C, q64, q32);
  return cudaGetLastError();
}

cudaError_t column_kinds(long long n, const uint8_t* is_int, int* kind, int* aux_of, cudaStream_t st) {
  if (n > 0) k_column_kinds<<<setup_grid(n, kSetupThreads), kSetupThreads, 0, st>>>(n, is_int, kind, aux_of);
  return cudaGetLastError();
}

// R = C = 1, then ruiz_iters Ruiz iterations (every factor of an iteration from the
// previous iteration's R and C) and the Pock-Chambolle step; each step writes the
// other buffer of a pair, and the result is copied back to R and C when it ends in
// R2 and C2.
cudaError_t launch_precondition(const DevSetup& s, int ruiz_iters, bool pock_chambolle, cudaStream_t st) {
  cudaError_t e = fill_f64(s.R, s.m, 1.0, st);
  if (e == cudaSuccess) e = fill_f64(s.C, s.n, 1.0, st);
  if (e != cudaSuccess) return e;
  double *r = s.R, *c = s.C, *r2 = s.R2, *c2 = s.C2;
  auto flip = [&] {
    double* t = r;
    r = r2;
    r2 = t;
    t = c;
    c = c2;
    c2 = t;
  };
  for (int it = 0; it < ruiz_iters; ++it) {
    side_factors<true>(s, r, c, r2, c2, st);
    flip();
  }
  if (pock_chambolle) {
    side_factors<false>(s, r, c, r2, c2, st);
    flip();
  }
  if (r != s.R) {
    if (s.m > 0) e = cudaMemcpyAsync(s.R, r, sizeof(double) * size_t(s.m), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.C, c, sizeof(double) * size_t(s.n), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t launch_scale_values(const DevSetup& s, cudaStream_t st) {
  const int gr = setup_grid(s.a_ntiles, kSetupThreads / 32), gc = setup_grid(s.t_ntiles, kSetupThreads / 32);
  k_scale_side<true><<<gr, kSetupThreads, 0, st>>>(s.a_tiles, s.a_ntiles, s.a_rowptr, s.a_cols, s.a_vals64,
                                                   s.a_vals32, s.R, s.C);
  k_scale_side<false><<<gc, kSetupThreads, 0, st>>>(s.t_tiles, s.t_ntiles, s.t_rowptr, s.t_cols, s.t_vals64,
                                                    s.t_vals32, s.C, s.R);
  return cudaGetLastError();
}

cudaError_t setup_norms(const DevSetup& s, const double* c64, const double* lo64, const double* hi64, cudaStream_t st,
                        SetupNorms* out) {
  const int g = s.red_blocks;
  k_setup_norms<<<g, kSetupThreads, 0, st>>>(s.a_vals64, s.nnz, c64, s.n, lo64, hi64, s.m, s.red);
  std::vector<double> h(4 * size_t(g));
  cudaError_t e = cudaMemcpyAsync(h.data(), s.red, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  SetupNorms r{0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < g; ++b) {
    r.amax = std::fmax(r.amax, h[4 * size_t(b)]);
    r.fro2 += h[4 * size_t(b) + 1];
    r.c2 += h[4 * size_t(b) + 2];
    r.q2 += h[4 * size_t(b) + 3];
  }
  *out = r;
  return cudaGetLastError();
}

}  // namespace scylla
