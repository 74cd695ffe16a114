// Bound propagation on the GPU (Section 2.3's activity-based tightening), in rounds:
// every active row computes, from the domains at the start of the round, the
// tightened bounds it implies for its columns (the arithmetic of one visit of the
// sequential propagation, in CSR order, one thread per row); then every column takes
// the largest proposed lower and the smallest proposed upper bound over its rows
// (read through the stored transpose; no atomics on the domains).  A row whose
// activity bounds already exclude [lo, hi], or that would empty a domain, is ignored
// from then on; a column whose merged proposals cross keeps its domain and counts a
// conflict.  The rows of the columns that changed are the next round's active rows.
// On integer data without ignored rows or conflicts this is the fixpoint of the
// sequential queue (the greatest fixpoint of a monotone tightening), bit for bit.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.h"

namespace scylla {

namespace {

constexpr int kPropThreads = 256;

int prop_grid(long long items) {
  long long g = (items + kPropThreads - 1) / kPropThreads;
  const long long cap = 8LL * device_sm_count();
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return int(g);
}

// position in A of every entry of the transpose: entry q of column j lies in row
// i = rows[q], whose column indices are ascending, so a binary search finds j
__global__ void k_prop_perm(int n, const int* __restrict__ t_rowptr, const int* __restrict__ t_rows,
                            const int* __restrict__ a_rowptr, const int* __restrict__ a_cols, int* __restrict__ perm) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    for (int q = t_rowptr[j]; q < t_rowptr[j + 1]; ++q) {
      const int i = t_rows[q];
      int lo = a_rowptr[i], hi = a_rowptr[i + 1] - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a_cols[mid] < j) lo = mid + 1;
        else hi = mid;
      }
      perm[q] = lo;
    }
  }
}

// one round's row visits.  state[i]: 0 no proposals this round, 1 proposals in
// plb/pub at the row's CSR positions (-inf / +inf where a bound is not tightened),
// 2 ignored for good
__global__ void __launch_bounds__(kPropThreads)
    k_prop_rows(PropDev P, const unsigned char* __restrict__ active) {
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.m; i += gridDim.x * blockDim.x) {
    if (P.state[i] == 2) continue;
    if (!active[i]) {
      P.state[i] = 0;
      continue;
    }
    const double lo_i = P.lo[i], hi_i = P.hi[i];
    if (lo_i == -inf && hi_i == inf) {
      P.state[i] = 0;
      continue;
    }
    const int p0 = P.rowptr[i], p1 = P.rowptr[i + 1];
    double minf = 0.0, maxf = 0.0;
    int nmin = 0, nmax = 0;
    for (int p = p0; p < p1; ++p) {
      const int j = P.cols[p];
      const double a = P.vals[p];
      const double bmin = a > 0.0 ? P.dl[j] : P.du[j];
      const double bmax = a > 0.0 ? P.du[j] : P.dl[j];
      if (isinf(bmin)) ++nmin;
      else minf = __dadd_rn(minf, __dmul_rn(a, bmin));
      if (isinf(bmax)) ++nmax;
      else maxf = __dadd_rn(maxf, __dmul_rn(a, bmax));
    }
    if ((nmin == 0 && hi_i != inf && minf > __dadd_rn(hi_i, 1e-9)) ||
        (nmax == 0 && lo_i != -inf && maxf < __dsub_rn(lo_i, 1e-9))) {
      P.state[i] = 2;
      continue;
    }
    bool ignore = false;
    for (int p = p0; p < p1; ++p) {
      const int j = P.cols[p];
      const double a = P.vals[p];
      const double old_lb = P.dl[j], old_ub = P.du[j];
      const double bmin = a > 0.0 ? old_lb : old_ub;
      const double bmax = a > 0.0 ? old_ub : old_lb;
      double rmin, rmax;
      if (isinf(bmin)) rmin = nmin == 1 ? minf : -inf;
      else rmin = nmin == 0 ? __dsub_rn(minf, __dmul_rn(a, bmin)) : -inf;
      if (isinf(bmax)) rmax = nmax == 1 ? maxf : inf;
      else rmax = nmax == 0 ? __dsub_rn(maxf, __dmul_rn(a, bmax)) : inf;
      double cand_lb = -inf, cand_ub = inf;
      if (hi_i != inf && rmin != -inf) {
        const double t = __ddiv_rn(__dsub_rn(hi_i, rmin), a);
        if (a > 0.0) cand_ub = t;
        else cand_lb = t;
      }
      if (lo_i != -inf && rmax != inf) {
        const double t = __ddiv_rn(__dsub_rn(lo_i, rmax), a);
        if (a > 0.0) cand_lb = t;
        else cand_ub = t;
      }
      double new_lb = old_lb, new_ub = old_ub;
      if (P.is_int[j]) {
        if (cand_ub != inf) {
          const double v = floor(__dadd_rn(cand_ub, 1e-6));
          if (v < old_ub) new_ub = v;
        }
        if (cand_lb != -inf) {
          const double v = ceil(__dsub_rn(cand_lb, 1e-6));
          if (v > old_lb) new_lb = v;
        }
      } else {
        if (cand_ub != inf &&
            (old_ub == inf || cand_ub < __dsub_rn(old_ub, __dmul_rn(1e-3, fmax(1.0, fabs(old_ub))))))
          new_ub = cand_ub;
        if (cand_lb != -inf &&
            (old_lb == -inf || cand_lb > __dadd_rn(old_lb, __dmul_rn(1e-3, fmax(1.0, fabs(old_lb))))))
          new_lb = cand_lb;
      }
      if (new_lb != old_lb || new_ub != old_ub) {
        if (new_lb > __dadd_rn(new_ub, 1e-9)) {
          ignore = true;
          break;
        }
      }
      P.plb[p] = new_lb != old_lb ? new_lb : -inf;
      P.pub[p] = new_ub != old_ub ? new_ub : inf;
    }
    P.state[i] = ignore ? 2 : 1;
  }
}

// the merge of one round: each column over its rows' proposals; changed columns
// mark their rows active for the next round.  count[0]: columns changed, count[1]:
// conflicts, count[2]: set when a row was marked
__global__ void __launch_bounds__(kPropThreads)
    k_prop_cols(PropDev P, unsigned char* __restrict__ active_next) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.n; j += gridDim.x * blockDim.x) {
    const int q0 = P.t_rowptr[j], q1 = P.t_rowptr[j + 1];
    const double ol = P.dl[j], ou = P.du[j];
    double nl = ol, nu = ou;
    for (int q = q0; q < q1; ++q) {
      const int i = P.t_rows[q];
      if (i >= P.m || P.state[i] != 1) continue;
      const int p = P.perm[q];
      nl = fmax(nl, P.plb[p]);
      nu = fmin(nu, P.pub[p]);
    }
    if (nl == ol && nu == ou) continue;
    if (nl > __dadd_rn(nu, 1e-9)) {
      atomicAdd(P.count + 1, 1ULL);
      continue;
    }
    P.dl[j] = nl;
    P.du[j] = nu;
    atomicAdd(P.count, 1ULL);
    bool marked = false;
    for (int q = q0; q < q1; ++q) {
      const int i = P.t_rows[q];
      if (i >= P.m || P.state[i] == 2) continue;
      active_next[i] = 1;
      marked = true;
    }
    if (marked) atomicOr(reinterpret_cast<unsigned long long*>(P.count + 2), 1ULL);
  }
}

}  // namespace

cudaError_t propagate_perm(int n, const int* t_rowptr, const int* t_rows, const int* a_rowptr, const int* a_cols,
                           int* perm, cudaStream_t st) {
  if (n > 0) k_prop_perm<<<prop_grid(n), kPropThreads, 0, st>>>(n, t_rowptr, t_rows, a_rowptr, a_cols, perm);
  return cudaGetLastError();
}

cudaError_t propagate_round(const PropDev& P, const unsigned char* active, unsigned char* active_next,
                            cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(active_next, 0, size_t(P.m > 0 ? P.m : 1), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.count, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (P.m > 0) k_prop_rows<<<prop_grid(P.m), kPropThreads, 0, st>>>(P, active);
  if (P.n > 0) k_prop_cols<<<prop_grid(P.n), kPropThreads, 0, st>>>(P, active_next);
  return cudaGetLastError();
}

}  // namespace scylla
