// Host side of the Scylla rounding step (arXiv 2307.03466, Section 2.3):
// fix-and-propagate, the exact MIP-feasibility test used by both success tests of
// Algorithm 1, and the perturbation used against cycling.
//
// Built with -ffp-contract=off so every floating-point operation rounds exactly as
// written; the fixings and domains are then reproducible bit for bit.
//
// Fix-and-propagate: the integer columns are visited in order of increasing
// distance |xbar_j - round(xbar_j)| (ties by index, round(v) = floor(v + 1/2)); one
// that propagation has already fixed is skipped, otherwise it is fixed to
// round(xbar_j) clamped to its domain and propagation runs.  Propagation is
// activity-based bound tightening with a FIFO queue of rows: a visit recomputes the
// row's minimum and maximum activity from scratch (finite parts in CSR order,
// infinite contributions counted) and derives, from the domains at the start of the
// visit, a bound for every column of the row.  Integer bounds are rounded inward
// with a 1e-6 tolerance and kept when strictly tighter; continuous bounds are kept
// when finite and tighter by more than 1e-3 max(1, |old|).  A row whose activity
// range misses [lo, hi] by more than 1e-9, or whose bounds would empty a domain, is
// ignored from then on (Section 2.3 keeps rounding past such a row by disregarding it)
// and changes nothing; otherwise its changes are applied together and the
// rows of each changed column are queued (ascending, unless queued or ignored).  One
// propagation stops after 20 m + 1000 row visits.  Finally every column takes its
// reference value projected onto its domain.
//
// The first propagation (every row queued once, before any fixing) depends only on
// the MIP, so its end state is kept in the handle and reused by later calls until the
// handle's bounds change.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "host_par.h"
#include "internal.h"
#include "lp_handle.h"

using namespace scylla;

namespace {

const double kInf = std::numeric_limits<double>::infinity();

struct Propagator {
  const scylla_lp& lp;

  // a column's domain, both bounds on one line
  struct Dom {
    double lb, ub;
  };
  std::vector<Dom> dom;

  // Everything a visit or a queue operation touches for row i, on one 64-byte line:
  // its bounds, its queue and ignored flags, and the activity data of its last full
  // visit (finite parts of the minimum and maximum activity, counts of unbounded
  // contributions, largest column span), kept current by every later bound change of
  // its columns (upd counts those updates).  The activity data only decides whether a
  // visit can end early; a visit that goes on recomputes everything from scratch in
  // CSR order.
  struct alignas(64) Row {
    double lo, hi;
    double minf, maxf, span;
    int32_t nmin, nmax, upd;
    uint8_t valid, inq, ignored;
  };
  std::vector<Row> rows;

  // FIFO of rows; a row is queued at most once (inq), so m slots suffice
  std::vector<int32_t> ring;
  int64_t head = 0, count = 0;

  explicit Propagator(const scylla_lp& h) : lp(h), dom(size_t(h.n0)), rows(size_t(h.m0)), ring(size_t(h.m0 > 0 ? h.m0 : 1)) {
    for (int64_t j = 0; j < h.n0; ++j) dom[size_t(j)] = Dom{h.l0[size_t(j)], h.u0[size_t(j)]};
    for (int64_t i = 0; i < h.m0; ++i) {
      Row& r = rows[size_t(i)];
      r = Row{};
      r.lo = h.lo0[size_t(i)];
      r.hi = h.hi0[size_t(i)];
    }
  }

  // continue from the end state of an earlier propagation (queue empty)
  Propagator(const scylla_lp& h, const std::vector<Dom>& d, const std::vector<Row>& r)
      : lp(h), dom(d), rows(r), ring(size_t(h.m0 > 0 ? h.m0 : 1)) {}

  void push(int32_t i) {
    Row& r = rows[size_t(i)];
    if (!r.inq && !r.ignored) {
      r.inq = 1;
      int64_t t = head + count;
      if (t >= lp.m0) t -= lp.m0;
      ring[size_t(t)] = i;
      ++count;
    }
  }

  int32_t pop() {
    const int32_t i = ring[size_t(head)];
    if (++head == lp.m0) head = 0;
    --count;
    return i;
  }

  // column j's domain moved from (ol, ou) to its current (tightened) one: update the
  // cached activity data of its rows (the span is left as an upper bound) and queue
  // them, in column order
  void tightened(int64_t j, double ol, double ou) {
    const double nl = dom[size_t(j)].lb, nu = dom[size_t(j)].ub;
    for (int64_t q = lp.colptr0[j]; q < lp.colptr0[j + 1]; ++q) {
      const int32_t i = lp.colrows0[q];
      Row& c = rows[size_t(i)];
      if (c.valid) {
        const double a = lp.colvals0[q];
        const double bo = a > 0 ? ol : ou, bn = a > 0 ? nl : nu;
        const double co = a > 0 ? ou : ol, cn = a > 0 ? nu : nl;
        if (bo != bn) {
          if (std::isinf(bo)) {
            c.nmin--;
            c.minf += a * bn;
          } else {
            c.minf += a * (bn - bo);
          }
        }
        if (co != cn) {
          if (std::isinf(co)) {
            c.nmax--;
            c.maxf += a * cn;
          } else {
            c.maxf += a * (cn - co);
          }
        }
        c.upd++;
      }
      push(i);
    }
  }

  // A side can tighten a bound only with exactly one unbounded contribution, or when
  // its slack (hi - minact, maxact - lo) is within the largest single-column span:
  // column j's candidate lies (slack - |a_j| (u_j - l_j)) / |a_j| beyond its own
  // bound.  True when both sides' slacks exceed the span by a relative margin of
  // 1e-6 (far above the rounding of the candidate arithmetic and of the cached sums,
  // which the integer rounding slack of 1e-6 and the continuous threshold of 1e-3
  // cover again): then no candidate can change a domain.
  static bool screened(double lo, double hi, double minf, double maxf, int nmin, int nmax, double span) {
    constexpr double kMarg = 1e-6;
    const bool hi_side =
        hi != kInf && (nmin == 1 || (nmin == 0 && !((hi - minf) > span * (1.0 + kMarg) +
                                                                   kMarg * (1.0 + std::fabs(hi) + std::fabs(minf)))));
    const bool lo_side =
        lo != -kInf && (nmax == 1 || (nmax == 0 && !((maxf - lo) > span * (1.0 + kMarg) +
                                                                     kMarg * (1.0 + std::fabs(lo) + std::fabs(maxf)))));
    return !hi_side && !lo_side;
  }

  struct Change {
    int64_t j;
    double lb, ub;
  };
  std::vector<Change> changes;  // of the row being visited (kept to reuse its storage)
  std::vector<Change> c_old;    // the same columns with their previous domains

  void visit(int32_t i) {
    Row& r = rows[size_t(i)];
    const double lo = r.lo, hi = r.hi;
    if (lo == -kInf && hi == kInf) return;
    // the cached data, at most 64 updates old (their rounding stays far below the
    // screen's margin), can end the visit without reading the row
    if (r.valid && r.upd < 64 && screened(lo, hi, r.minf, r.maxf, r.nmin, r.nmax, r.span)) return;
    const int64_t p0 = lp.rowptr0[i], p1 = lp.rowptr0[i + 1];
    double minf = 0.0, maxf = 0.0;
    double span = 0.0;  // largest |a_j| (u_j - l_j) of the row (+inf with an unbounded domain)
    int nmin = 0, nmax = 0;
    for (int64_t p = p0; p < p1; ++p) {
      const int64_t j = lp.cols0[p];
      const double a = lp.vals0[p];
      const Dom d = dom[size_t(j)];
      const double bmin = a > 0 ? d.lb : d.ub;
      const double bmax = a > 0 ? d.ub : d.lb;
      if (std::isinf(bmin)) nmin++;
      else minf += a * bmin;
      if (std::isinf(bmax)) nmax++;
      else maxf += a * bmax;
      span = std::max(span, std::fabs(a) * (d.ub - d.lb));
    }
    if (nmin == 0 && hi != kInf && minf > hi + 1e-9) {
      r.ignored = 1;
      return;
    }
    if (nmax == 0 && lo != -kInf && maxf < lo - 1e-9) {
      r.ignored = 1;
      return;
    }
    r.minf = minf;
    r.maxf = maxf;
    r.span = span;
    r.nmin = nmin;
    r.nmax = nmax;
    r.upd = 0;
    r.valid = 1;
    if (screened(lo, hi, minf, maxf, nmin, nmax, span)) return;  // no candidate can change a domain
    changes.clear();
    for (int64_t p = p0; p < p1; ++p) {
      const int64_t j = lp.cols0[p];
      const double a = lp.vals0[p];
      const Dom d = dom[size_t(j)];
      const double bmin = a > 0 ? d.lb : d.ub;
      const double bmax = a > 0 ? d.ub : d.lb;
      double rmin, rmax;
      if (std::isinf(bmin)) rmin = (nmin == 1) ? minf : -kInf;
      else rmin = (nmin == 0) ? (minf - a * bmin) : -kInf;
      if (std::isinf(bmax)) rmax = (nmax == 1) ? maxf : kInf;
      else rmax = (nmax == 0) ? (maxf - a * bmax) : kInf;
      double cand_lb = -kInf, cand_ub = kInf;
      if (hi != kInf && rmin != -kInf) {
        const double t = (hi - rmin) / a;
        if (a > 0) cand_ub = t;
        else cand_lb = t;
      }
      if (lo != -kInf && rmax != kInf) {
        const double t = (lo - rmax) / a;
        if (a > 0) cand_lb = t;
        else cand_ub = t;
      }
      const double old_lb = d.lb, old_ub = d.ub;
      double nlb = old_lb, nub = old_ub;
      if (lp.int0[j]) {
        if (cand_ub != kInf) {
          const double v = std::floor(cand_ub + 1e-6);
          if (v < old_ub) nub = v;
        }
        if (cand_lb != -kInf) {
          const double v = std::ceil(cand_lb - 1e-6);
          if (v > old_lb) nlb = v;
        }
      } else {
        if (cand_ub != kInf && (old_ub == kInf || cand_ub < old_ub - 1e-3 * std::max(1.0, std::fabs(old_ub))))
          nub = cand_ub;
        if (cand_lb != -kInf && (old_lb == -kInf || cand_lb > old_lb + 1e-3 * std::max(1.0, std::fabs(old_lb))))
          nlb = cand_lb;
      }
      if (nlb == old_lb && nub == old_ub) continue;
      if (nlb > nub + 1e-9) {
        r.ignored = 1;
        return;
      }
      changes.push_back({j, nlb, nub});
    }
    // all changes are applied before any row is queued or its cache updated; both only
    // read the new domains, so doing them column by column keeps the queue order
    for (const Change& c : changes) {
      Dom& d = dom[size_t(c.j)];
      const double ol = d.lb, ou = d.ub;
      d.lb = c.lb;
      d.ub = c.ub;
      c_old.push_back({c.j, ol, ou});
    }
    for (const Change& c : c_old) tightened(c.j, c.lb, c.ub);
    c_old.clear();
  }

  void run() {
    const int64_t cap = 20 * lp.m0 + 1000;
    int64_t visits = 0;
    while (count > 0) {
      const int32_t i = pop();
      rows[size_t(i)].inq = 0;
      if (rows[size_t(i)].ignored) continue;
      if (visits >= cap) {
        while (count > 0) rows[size_t(pop())].inq = 0;
        break;
      }
      ++visits;
      visit(i);
    }
  }
};

// the end state of the first propagation of the handle's MIP, computed on first use
struct RootState {
  std::vector<Propagator::Dom> dom;
  std::vector<Propagator::Row> rows;
};

const RootState& root_state(const scylla_lp& lp) {
  if (!lp.root_prop) {
    Propagator pr(lp);
    for (int32_t i = 0; i < lp.m0; ++i) pr.push(i);
    pr.run();
    auto st = std::make_shared<RootState>();
    st->dom = std::move(pr.dom);
    st->rows = std::move(pr.rows);
    lp.root_prop = st;
  }
  return *std::static_pointer_cast<const RootState>(lp.root_prop);
}

inline double round_half_up(double v) { return std::floor(v + 0.5); }

bool is_int_value(double v) { return std::isfinite(v) && v == std::floor(v) && std::fabs(v) < 140737488355328.0; }

// Neumaier's compensated sum of a_p x_p in CSR order
double neumaier_row(const scylla_lp& lp, int64_t i, const double* x) {
  double s = 0.0, comp = 0.0;
  for (int64_t p = lp.rowptr0[i]; p < lp.rowptr0[i + 1]; ++p) {
    const double t = lp.vals0[p] * x[lp.cols0[p]];
    const double tt = s + t;
    if (std::fabs(s) >= std::fabs(t)) comp += (s - tt) + t;
    else comp += (t - tt) + s;
    s = tt;
  }
  return s + comp;
}

}  // namespace

namespace scylla {

// exact feasibility test (Algorithm 1, "MIP-feasible"): integrality exact; rows with
// integer coefficients, bounds and column values (|v| < 2^47) in exact 128-bit
// integer arithmetic (each product is below 2^94 and a row has fewer than 2^31
// entries, so a sum stays below 2^125 and cannot overflow); other rows by compensated FP64 sums with tolerance
// 1e-6 max(1, |bound|); continuous column bounds with the same tolerance.
bool check_feasible_host(const scylla_lp& lp, const double* x) {
  const double tol = 1e-6;
  for (int64_t j = 0; j < lp.n0; ++j) {
    const double v = x[j];
    if (!std::isfinite(v)) return false;
    if (lp.int0[j]) {
      if (v != std::floor(v) || v < lp.l0[j] || v > lp.u0[j]) return false;
    } else {
      if (v < lp.l0[j] - tol * std::max(1.0, std::fabs(lp.l0[j])) ||
          v > lp.u0[j] + tol * std::max(1.0, std::fabs(lp.u0[j])))
        return false;
    }
  }
  for (int64_t i = 0; i < lp.m0; ++i) {
    const double lo = lp.lo0[i], hi = lp.hi0[i];
    bool exact = (lo == -kInf || is_int_value(lo)) && (hi == kInf || is_int_value(hi));
    for (int64_t p = lp.rowptr0[i]; exact && p < lp.rowptr0[i + 1]; ++p)
      exact = is_int_value(lp.vals0[p]) && is_int_value(x[lp.cols0[p]]);
    if (exact) {
      __int128 act = 0;
      for (int64_t p = lp.rowptr0[i]; p < lp.rowptr0[i + 1]; ++p)
        act += (__int128)(int64_t)lp.vals0[p] * (__int128)(int64_t)x[lp.cols0[p]];
      if (lo != -kInf && act < (__int128)(int64_t)lo) return false;
      if (hi != kInf && act > (__int128)(int64_t)hi) return false;
    } else {
      const double act = neumaier_row(lp, i, x);
      if (lo != -kInf && act < lo - tol * std::max(1.0, std::fabs(lo))) return false;
      if (hi != kInf && act > hi + tol * std::max(1.0, std::fabs(hi))) return false;
    }
  }
  return true;
}

}  // namespace scylla

namespace {

// the fixing loop for one point, from the kept first propagation (read only, so that
// several points can run at once)
void fix_one(const scylla_lp& lp, const RootState& root, const double* xbar, double* xhat, double* dom_lo,
             double* dom_hi, int32_t* fixed_cols, int64_t* n_fixed, uint8_t* ignored_rows) {
  Propagator pr(lp, root.dom, root.rows);
  std::vector<int64_t> order;
  order.reserve(size_t(lp.n_int));
  std::vector<double> dist(size_t(lp.n0), 0.0);
  for (int64_t j = 0; j < lp.n0; ++j) {
    if (!lp.int0[j]) continue;
    order.push_back(j);
    dist[j] = std::fabs(xbar[j] - round_half_up(xbar[j]));
  }
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    if (dist[a] != dist[b]) return dist[a] < dist[b];
    return a < b;
  });
  int64_t nf = 0;
  for (int64_t j : order) {
    Propagator::Dom& d = pr.dom[size_t(j)];
    if (d.lb == d.ub) continue;
    double v = round_half_up(xbar[j]);
    v = std::min(std::max(v, d.lb), d.ub);
    const double ol = d.lb, ou = d.ub;
    d.lb = v;
    d.ub = v;
    if (fixed_cols) fixed_cols[nf] = int32_t(j);
    ++nf;
    pr.tightened(j, ol, ou);
    pr.run();
  }
  for (int64_t j = 0; j < lp.n0; ++j) {
    const Propagator::Dom d = pr.dom[size_t(j)];
    xhat[j] = std::min(std::max(xbar[j], d.lb), d.ub);
    if (dom_lo) dom_lo[j] = d.lb;
    if (dom_hi) dom_hi[j] = d.ub;
  }
  if (n_fixed) *n_fixed = nf;
  if (ignored_rows)
    for (int64_t i = 0; i < lp.m0; ++i) ignored_rows[i] = pr.rows[size_t(i)].ignored;
}

}  // namespace

namespace scylla {

int fix_and_propagate_host(const scylla_lp& lp, const double* xbar, double* xhat, double* dom_lo, double* dom_hi,
                           int32_t* fixed_cols, int64_t* n_fixed, uint8_t* ignored_rows) {
  const int rc = lp.ensure_host_matrix();
  if (rc != SCYLLA_OK) return rc;
  lp.ensure_columns();
  fix_one(lp, root_state(lp), xbar, xhat, dom_lo, dom_hi, fixed_cols, n_fixed, ignored_rows);
  return SCYLLA_OK;
}

// K points at once: the set-up (host copies, transpose, first propagation) on the
// calling thread, then the points dealt round-robin to the host threads, each with a
// private copy of the kept state; point k gives what fix_and_propagate_host gives
int fix_and_propagate_many_host(const scylla_lp& lp, int64_t K, const double* xbar, double* xhat, double* dom_lo,
                                double* dom_hi, int64_t* n_fixed) {
  const int rc = lp.ensure_host_matrix();
  if (rc != SCYLLA_OK) return rc;
  lp.ensure_columns();
  const RootState& root = root_state(lp);
  const int T = int(std::max<int64_t>(1, std::min<int64_t>(K, host_threads())));
  const size_t n = size_t(lp.n0);
  std::atomic<bool> oom{false};
  fork_join(T, [&](int t) {
    try {
      for (int64_t k = t; k < K && !oom.load(); k += T)
        fix_one(lp, root, xbar + size_t(k) * n, xhat + size_t(k) * n, dom_lo ? dom_lo + size_t(k) * n : nullptr,
                dom_hi ? dom_hi + size_t(k) * n : nullptr, nullptr, n_fixed ? n_fixed + k : nullptr, nullptr);
    } catch (const std::bad_alloc&) {
      oom = true;
    }
  });
  if (oom) throw std::bad_alloc();
  return SCYLLA_OK;
}

// SplitMix64 (Steele, Lea, Flood 2014)
struct SplitMix64 {
  uint64_t s;
  explicit SplitMix64(uint64_t seed) : s(seed) {}
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return double(next() >> 11) * 0x1.0p-53; }
};

// one unit toward xbar, or away from it when v already is round(xbar); the other
// direction when the first leaves [l, u]
static double flip_value(double v, double xb, double l, double u) {
  const double r = std::floor(xb + 0.5);
  double s = xb >= v ? 1.0 : -1.0;
  if (v == r) s = -s;
  const double d[2] = {s, -s};
  for (double dd : d) {
    const double w = v + dd;
    if (l <= w && w <= u) return w;
  }
  return v;
}

// Section 2.3 (after Fischetti-Glover-Lodi 2005).  kind 1 (short cycle): flip the TT
// integer columns with largest |xbar - xhat| > 0, TT ~ U{10..30}; if there is none, or
// kind 2 (long cycle): flip column j when |xbar_j - xhat_j| + max(rho_j, 0) > 0.5,
// rho_j ~ U[-0.3, 0.7] drawn in ascending j.  The stream is SplitMix64(seed ^ K).
int64_t perturb_host(const scylla_lp& lp, double* x, const double* xbar, int kind, int64_t K, uint64_t seed) {
  SplitMix64 rng(seed ^ uint64_t(K));
  int64_t flipped = 0;
  if (kind == 1) {
    const int64_t TT = 10 + int64_t(std::floor(rng.uniform() * 21.0));
    std::vector<std::pair<double, int64_t>> cand;
    for (int64_t j = 0; j < lp.n0; ++j) {
      if (!lp.int0[j]) continue;
      const double sv = std::fabs(xbar[j] - x[j]);
      if (sv > 0) cand.push_back({sv, j});
    }
    if (!cand.empty()) {
      std::stable_sort(cand.begin(), cand.end(), [](const std::pair<double, int64_t>& a,
                                                   const std::pair<double, int64_t>& b) {
        if (a.first != b.first) return a.first > b.first;
        return a.second < b.second;
      });
      const int64_t cnt = std::min<int64_t>(TT, int64_t(cand.size()));
      for (int64_t q = 0; q < cnt; ++q) {
        const int64_t j = cand[q].second;
        const double w = flip_value(x[j], xbar[j], lp.l0[j], lp.u0[j]);
        flipped += (w != x[j]);
        x[j] = w;
      }
      return flipped;
    }
  }
  for (int64_t j = 0; j < lp.n0; ++j) {
    if (!lp.int0[j]) continue;
    const double rho = -0.3 + rng.uniform();
    if (std::fabs(xbar[j] - x[j]) + std::max(rho, 0.0) > 0.5) {
      const double w = flip_value(x[j], xbar[j], lp.l0[j], lp.u0[j]);
      flipped += (w != x[j]);
      x[j] = w;
    }
  }
  return flipped;
}

}  // namespace scylla

extern "C" int scylla_fix_and_propagate(const scylla_lp* lp, const double* xbar, double* xhat, double* dom_lo,
                                        double* dom_hi, int32_t* fixed_cols, int64_t* n_fixed,
                                        uint8_t* ignored_rows) {
  if (!lp || !xbar || !xhat) {
    set_error("null argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  for (int64_t j = 0; j < lp->n0; ++j)
    if (std::isnan(xbar[j])) {
      set_error("xbar has NaN at " + std::to_string(j));
      return SCYLLA_ERR_INVALID_ARG;
    }
  try {
    return fix_and_propagate_host(*lp, xbar, xhat, dom_lo, dom_hi, fixed_cols, n_fixed, ignored_rows);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return SCYLLA_ERR_OOM;
  }
}

extern "C" int scylla_fix_and_propagate_many(const scylla_lp* lp, int32_t K, const double* xbar, double* xhat,
                                             double* dom_lo, double* dom_hi, int64_t* n_fixed) {
  if (!lp || K < 0 || (K > 0 && (!xbar || !xhat))) {
    set_error("invalid argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  const int64_t total = int64_t(K) * lp->n0;
  for (int64_t q = 0; q < total; ++q)
    if (std::isnan(xbar[q])) {
      set_error("xbar has NaN at point " + std::to_string(q / lp->n0) + ", column " + std::to_string(q % lp->n0));
      return SCYLLA_ERR_INVALID_ARG;
    }
  try {
    return fix_and_propagate_many_host(*lp, K, xbar, xhat, dom_lo, dom_hi, n_fixed);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return SCYLLA_ERR_OOM;
  }
}

extern "C" int scylla_check_feasible(const scylla_lp* lp, const double* x, int32_t* feasible) {
  if (!lp || !x || !feasible) {
    set_error("null argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  try {
    const int rc = lp->ensure_host_matrix();
    if (rc != SCYLLA_OK) return rc;
    *feasible = check_feasible_host(*lp, x) ? 1 : 0;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return SCYLLA_ERR_OOM;
  }
  return SCYLLA_OK;
}

extern "C" int scylla_perturb(const scylla_lp* lp, double* xhat, const double* xbar, int32_t kind, int64_t K,
                              uint64_t seed, int64_t* flipped) {
  if (!lp || !xhat || !xbar || (kind != 1 && kind != 2)) {
    set_error("invalid argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  try {
    const int rv = lp->ensure_host_vectors();
    if (rv != SCYLLA_OK) return rv;
    const int64_t f = perturb_host(*lp, xhat, xbar, kind, K, seed);
    if (flipped) *flipped = f;
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return SCYLLA_ERR_OOM;
  }
  return SCYLLA_OK;
}
