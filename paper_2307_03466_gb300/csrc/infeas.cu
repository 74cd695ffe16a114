// Infeasibility detection during a single-LP solve.  Scylla hands its LP
// relaxations to PDLP (Section 2.1), whose solver also reports relaxations without a
// feasible point; a report of that kind rests on a dual ray y with D(y) > 0, where
//     D(y) = sum_i min_{lo_i <= s_i <= hi_i} y_i s_i  -  sum_j max_{l_j <= x_j <= u_j} (A^T y)_j x_j
// (weak duality: every feasible x has first sum <= y^T A x = (A^T y)^T x <= second sum).
// On an infeasible LP the PDHG dual iterates drift along such a ray, so the change
// of y between two checks is the candidate.
//
// At the check after k = q n_check attempts:
//   * q >= 2 tests the candidate y_k - y_a, y_a being y at the last earlier check
//     whose q was a power of two, with every entry set to 0 whose sign would need an
//     infinite row bound;
//   * q a power of two then makes y_k the anchor y_a of the following checks.
// Both run in the scaled space the solve iterates in (y~ = y / R, lo~ = R lo,
// A~ = R A C, [l~, u~] = [l, u] / C), where every term of D equals the unscaled one.
// The two kernels below sit between the column and the row halves of the check; the
// row half's decision ends the solve SCYLLA_INFEASIBLE when D > kInfeasMargin S,
// S being the sum of the absolute values of D's terms.  Sums over rows and columns
// are FP64 block reductions in a fixed order (their rounding is a few ulps of S);
// each (A~^T y)_j is a compensated sum over the column's entries in row order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "device_common.cuh"

namespace scylla {

namespace {

// q of this check when it tests or moves the anchor, else 0 (the start point's check
// and one at an iteration limit between multiples of n_check do neither)
__device__ __forceinline__ long long check_index(long long k, int nc) {
  return (k >= nc && k % nc == 0) ? k / nc : 0;
}

__device__ __forceinline__ void pdl_wait_then_trigger() {
  cudaGridDependencySynchronize();
  cudaTriggerProgrammaticLaunchCompletion();
}

// the candidate ray and the row terms of D: y~_i - y~a_i, kept where its sign has a
// finite row bound, and its smallest product with [lo~_i, hi~_i]; the anchor moves
// when q is a power of two
template <typename T>
__global__ void __launch_bounds__(kThreads) k_infeas_rows(DevLP<T> d) {
  const Control* ctl = d.ctl;
  pdl_wait_then_trigger();
  if (ctl->done) return;
  const long long q = check_index(ctl->k, d.n_check);
  if (q == 0) return;
  const bool test = q >= 2, move = (q & (q - 1)) == 0;
  const T* __restrict__ y = d.Y[ctl->ix_cur];
  double acc[kNIR] = {0.0, 0.0};
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) {
    const T yi = y[i];
    if (test) {
      double c = to_f64(yi) - to_f64(d.inf_anchor[i]);
      double t = 0.0;
      if (c > 0.0) {
        const double lo = d.lo64[i];
        if (above_neg_inf(lo)) t = c * lo;
        else c = 0.0;
      } else if (c < 0.0) {
        const double hi = d.hi64[i];
        if (below_pos_inf(hi)) t = c * hi;
        else c = 0.0;
      }
      d.inf_cand[i] = c;
      acc[0] += t;
      acc[1] += fabs(t);
    }
    if (move) d.inf_anchor[i] = yi;
  }
  block_store_partials<kNIR>(acc, d.inf_part);
}

// Neumaier's compensated running sum
struct Comp {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double t) {
    const double u = s + t;
    c += fabs(s) >= fabs(t) ? (s - u) + t : (t - u) + s;
    s = u;
  }
};

// the column terms of D: r_j = (A~^T cand)_j and its largest product with
// [l~_j, u~_j] (counted as infinite when that bound is); the last block reduces both
// kernels' partials and hands D and S to the check's decision
template <typename T>
__global__ void __launch_bounds__(kThreads) k_infeas_cols(DevLP<T> d) {
  Control* ctl = d.ctl;
  pdl_wait_then_trigger();
  if (ctl->done) return;
  if (check_index(ctl->k, d.n_check) < 2) return;
  double acc[kNIC] = {0.0, 0.0, 0.0};
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride) {
    Comp r;
    const int p1 = d.t_rowptr[j + 1];
    for (int p = d.t_rowptr[j]; p < p1; ++p) r.add(d.t_vals64[p] * d.inf_cand[d.t_cols[p]]);
    const double rj = r.s + r.c;
    double t = 0.0;
    if (rj > 0.0) {
      const double u = d.u64[j];
      if (below_pos_inf(u)) t = rj * u;
      else acc[2] += 1.0;
    } else if (rj < 0.0) {
      const double l = d.l64[j];
      if (above_neg_inf(l)) t = rj * l;
      else acc[2] += 1.0;
    }
    acc[0] += t;
    acc[1] += fabs(t);
  }
  const int G = d.inf_grid;
  block_store_partials<kNIC>(acc, d.inf_part + kNIR * G);
  if (!is_last_block(&ctl->cnt_inf)) return;
  __shared__ double scratch[(kNIR + kNIC) * (kThreads - 32)];
  __shared__ double red[kNIR + kNIC];
  reduce_two<kNIR, kNIC>(d.inf_part, G, d.inf_part + kNIR * G, G, scratch, red);
  if (threadIdx.x == 0) {
    // D = (row terms) - (column terms); a term that needs an infinite bound makes it -inf
    ctl->inf_gap = red[kNIR + 2] > 0.0 ? -INFINITY : red[0] - red[kNIR];
    ctl->inf_scale = red[1] + red[kNIR + 1];
    ctl->inf_tested = 1;
    ctl->cnt_inf = 0;
  }
}

template <typename T>
__global__ void k_get_cert(DevLP<T> d, double* out, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = d.inf_cand[i] * d.R[i];
}

template <typename T>
cudaError_t launch_pdl(void (*kernel)(DevLP<T>), int grid, const DevLP<T>& d, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = d.pdl ? attr : nullptr;
  cfg.numAttrs = d.pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, d);
}

}  // namespace

template <typename T>
cudaError_t launch_infeas(const DevLP<T>& d, cudaStream_t st) {
  cudaError_t e = launch_pdl<T>(k_infeas_rows<T>, d.inf_grid, d, st);
  if (e == cudaSuccess) e = launch_pdl<T>(k_infeas_cols<T>, d.inf_grid, d, st);
  return e;
}

template <typename T>
cudaError_t launch_get_cert(const DevLP<T>& d, double* out, int count, cudaStream_t st) {
  int g = (count + kThreads - 1) / kThreads;
  g = g < 1 ? 1 : (g > 1024 ? 1024 : g);
  k_get_cert<T><<<g, kThreads, 0, st>>>(d, out, count);
  return cudaGetLastError();
}

template cudaError_t launch_infeas<float>(const DevLP<float>&, cudaStream_t);
template cudaError_t launch_infeas<double>(const DevLP<double>&, cudaStream_t);
template cudaError_t launch_get_cert<float>(const DevLP<float>&, double*, int, cudaStream_t);
template cudaError_t launch_get_cert<double>(const DevLP<double>&, double*, int, cudaStream_t);

}  // namespace scylla
