// scylla_run: the outer loop of Scylla (arXiv 2307.03466, Algorithm 1).
//
//   K = 1, eps = eps1, c_hat = c
//   while limits not reached:
//     PDHG on the GPU until relative KKT <= eps (or iteration limit / stalling)
//     if round(xbar) is MIP-feasible and xbar was within 1e-6 of it: return it
//     xhat = fix-and-propagate(xbar)             (host, Section 2.3)
//     if xhat is MIP-feasible: return it
//     (optional) re-solve the continuous part with xhat's integers fixed; if
//       that point is MIP-feasible: return it
//     if xhat repeats an earlier rounding: perturb it (Section 2.3)
//     objective update around xhat for round K   (GPU, Section 2.4)
//     eps = max(beta eps, eps_floor); K = K + 1   (Section 2.2)
//   return nothing found
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "internal.h"
#include "lp_handle.h"

namespace scylla {
int fix_and_propagate_host(const scylla_lp& lp, const double* xbar, double* xhat, double* dom_lo, double* dom_hi,
                           int32_t* fixed_cols, int64_t* n_fixed, uint8_t* ignored_rows);
int64_t perturb_host(const scylla_lp& lp, double* x, const double* xbar, int kind, int64_t K, uint64_t seed);
}  // namespace scylla

using namespace scylla;

static int run_impl(scylla_lp* lp, double* x_out, scylla_run_result* out);

extern "C" int scylla_run(scylla_lp* lp, double* x_out, scylla_run_result* out) {
  if (!lp || !x_out || !out) {
    set_error("null argument");
    return SCYLLA_ERR_INVALID_ARG;
  }
  try {
    return run_impl(lp, x_out, out);
  } catch (const std::bad_alloc&) {
    set_error("host allocation failed");
    return SCYLLA_ERR_OOM;
  }
}

static int run_impl(scylla_lp* lp, double* x_out, scylla_run_result* out) {
  std::memset(out, 0, sizeof(*out));
  out->status = SCYLLA_NOT_FOUND;
  {
    const int rc = lp->ensure_host_matrix();  // the propagation and the feasibility test read it
    if (rc != SCYLLA_OK) return rc;
  }
  const auto t0 = std::chrono::steady_clock::now();
  auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  const scylla_params& p = lp->p;
  const int64_t n = lp->n0;
  std::vector<double> xbar(n), xr(n), xhat(n);
  std::vector<int64_t> int_cols;
  for (int64_t j = 0; j < n; ++j)
    if (lp->int0[j]) int_cols.push_back(j);
  std::vector<std::vector<double>> history;
  std::set<std::vector<double>> seen;
  double eps = p.eps1;
  int64_t total = 0;
  int64_t K = 1;
  auto finish = [&](const std::vector<double>& x, int by) {
    std::memcpy(x_out, x.data(), sizeof(double) * n);
    out->status = SCYLLA_FOUND;
    out->found_by = by;
    double obj = 0.0;
    for (int64_t j = 0; j < n; ++j) obj += lp->c0[j] * x[j];
    out->objective = obj;
  };
  int rc = SCYLLA_OK;
  for (; K <= p.max_rounds && total < p.total_iter_cap; ++K) {
    if (p.time_limit_s > 0 && elapsed() > p.time_limit_s) {
      rc = SCYLLA_ERR_TIMEOUT;
      set_error("time limit reached");
      break;
    }
    scylla_pdhg_result res;
    const int64_t lim = std::min<int64_t>(p.iter_limit, p.total_iter_cap - total);
    rc = lp->solve(eps, lim, p.run_stall_checks, &res);
    if (rc != SCYLLA_OK) break;
    total += res.iterations;
    out->seconds_pdhg += res.seconds;
    rc = lp->fetch_x(xbar.data(), int(n));
    if (rc != SCYLLA_OK) break;
    auto tf = std::chrono::steady_clock::now();
    // Algorithm 1: is the PDHG point itself MIP-feasible (after rounding)?
    bool near = true;
    xr = xbar;
    for (int64_t j : int_cols) {
      const double r = std::floor(xbar[j] + 0.5);
      if (std::fabs(xbar[j] - r) > 1e-6) near = false;
      xr[j] = r;
    }
    if (near && check_feasible_host(*lp, xr.data())) {
      out->seconds_fixprop += std::chrono::duration<double>(std::chrono::steady_clock::now() - tf).count();
      finish(xr, 1);
      out->rounds = K;
      break;
    }
    fix_and_propagate_host(*lp, xbar.data(), xhat.data(), nullptr, nullptr, nullptr, nullptr, nullptr);
    if (check_feasible_host(*lp, xhat.data())) {
      out->seconds_fixprop += std::chrono::duration<double>(std::chrono::steady_clock::now() - tf).count();
      finish(xhat, 2);
      out->rounds = K;
      break;
    }
    // continuous repair of the fix-and-propagate point (an extension; off by default)
    if (p.repair_iters > 0) {
      out->seconds_fixprop += std::chrono::duration<double>(std::chrono::steady_clock::now() - tf).count();
      scylla_repair_result rr;
      std::memset(&rr, 0, sizeof(rr));
      rc = lp->repair(xhat.data(), p.repair_tol, std::min<int64_t>(p.repair_iters, p.total_iter_cap - total),
                      xr.data(), &rr);
      if (rc != SCYLLA_OK) break;
      total += rr.iterations;
      out->seconds_pdhg += rr.seconds;
      if (rr.status == SCYLLA_FOUND) {
        finish(xr, 3);
        out->rounds = K;
        break;
      }
      tf = std::chrono::steady_clock::now();  // the cycle handling's time follows
    }
    // cycle test on the integer part
    std::vector<double> key(int_cols.size());
    for (size_t q = 0; q < int_cols.size(); ++q) key[q] = xhat[int_cols[q]];
    int kind = 0;
    if (!history.empty()) {
      if (key == history.back()) kind = 1;
      else if (seen.count(key)) kind = 2;
    }
    if (kind) {
      perturb_host(*lp, xhat.data(), xbar.data(), kind, K, p.seed);
      out->perturbations++;
      for (size_t q = 0; q < int_cols.size(); ++q) key[q] = xhat[int_cols[q]];
    }
    out->seconds_fixprop += std::chrono::duration<double>(std::chrono::steady_clock::now() - tf).count();
    if (!history.empty()) seen.insert(history.back());
    history.push_back(key);
    rc = lp->set_objective(xhat.data(), int32_t(K));
    if (rc != SCYLLA_OK) break;
    eps = std::max(p.beta * eps, p.eps_floor);
  }
  if (out->status != SCYLLA_FOUND) out->rounds = std::min<int64_t>(K, p.max_rounds);
  out->total_iterations = total;
  out->seconds = elapsed();
  return rc;
}
