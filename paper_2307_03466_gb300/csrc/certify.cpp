// Host test of a certificate of infeasibility of the original LP relaxation
//     lo <= A x <= hi,   l <= x <= u
// by weak duality.  Scylla hands its LP solves to PDLP (Section 2.1), whose solver also
// reports relaxations without a feasible point; a report of that kind rests on a dual
// ray y with D(y) > 0, where
//     D(y) = sum_i min_{lo_i <= s_i <= hi_i} y_i s_i  -  sum_j max_{l_j <= x_j <= u_j} (A^T y)_j x_j,
// because every feasible x has (first sum) <= y^T A x = (A^T y)^T x <= (second sum).
// A term that needs an infinite bound makes D(y) = -inf (that y proves nothing).  All
// sums are Neumaier-compensated FP64 in a fixed order (rows ascending; each column's
// entries in row order through the stored transpose), so the value is reproducible.
#include <cmath>
#include <cstdint>
#include <limits>
#include <new>
#include <string>

#include "internal.h"
#include "lp_handle.h"

namespace {

const double kInf = std::numeric_limits<double>::infinity();

// Neumaier's compensated running sum
struct CompSum {
  double s = 0.0, c = 0.0;
  void add(double t) {
    const double tt = s + t;
    if (std::fabs(s) >= std::fabs(t)) c += (s - tt) + t;
    else c += (t - tt) + s;
    s = tt;
  }
  double value() const { return s + c; }
};

}  // namespace

namespace scylla {

double farkas_gap_host(const scylla_lp& lp, const double* y) {
  CompSum left;
  for (int64_t i = 0; i < lp.m0; ++i) {
    const double yi = y[i];
    if (yi > 0.0) {
      if (lp.lo0[size_t(i)] == -kInf) return -kInf;
      left.add(yi * lp.lo0[size_t(i)]);
    } else if (yi < 0.0) {
      if (lp.hi0[size_t(i)] == kInf) return -kInf;
      left.add(yi * lp.hi0[size_t(i)]);
    }
  }
  CompSum right;
  for (int64_t j = 0; j < lp.n0; ++j) {
    CompSum r;
    for (int64_t q = lp.colptr0[size_t(j)]; q < lp.colptr0[size_t(j) + 1]; ++q)
      r.add(lp.colvals0[size_t(q)] * y[lp.colrows0[size_t(q)]]);
    const double rj = r.value();
    if (rj > 0.0) {
      if (lp.u0[size_t(j)] == kInf) return -kInf;
      right.add(rj * lp.u0[size_t(j)]);
    } else if (rj < 0.0) {
      if (lp.l0[size_t(j)] == -kInf) return -kInf;
      right.add(rj * lp.l0[size_t(j)]);
    }
  }
  return left.value() - right.value();
}

}  // namespace scylla

extern "C" int scylla_farkas_gap(const scylla_lp* lp, const double* y, double* gap) {
  if (!lp || !gap || (!y && lp->m0 > 0)) {
    scylla::set_error("null argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < lp->m0; ++i)
    if (!std::isfinite(y[i])) {
      scylla::set_error("y not finite at row " + std::to_string(i));
      return SCYLLA_ERR_INVALID_ARG;
    }
  try {
    const int rc = lp->ensure_host_matrix();
    if (rc != SCYLLA_OK) return rc;
    lp->ensure_columns();
    *gap = scylla::farkas_gap_host(*lp, y);
  } catch (const std::bad_alloc&) {
    scylla::set_error("host allocation failed");
    return SCYLLA_ERR_OOM;
  }
  return SCYLLA_OK;
}
