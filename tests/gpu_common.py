"""Shared helpers of the GPU parity tests: build the library once, create matching
GPU and oracle LPs from the same seeded instance, and compare iterates."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg as O
from paper_2307_03466_gb300 import instances as I

torch = pytest.importorskip("torch")

INF = np.inf
TOL = 1e-9        # FP64 iterates against the oracle
TOL_LONG = 2e-6   # adaptive runs of 1000 attempts on the device's decisions (worst seen 1.24e-6)


def gpu_available() -> bool:
    return bool(torch.cuda.is_available())


def lib():
    from paper_2307_03466_gb300 import build as B
    from paper_2307_03466_gb300 import scylla as S
    B.build()
    S.lib()
    return S


PDHG_KEYS = ("n_check", "ruiz_iters", "pock_chambolle", "adaptive_step", "restarts", "primal_weight_update",
             "fixed_step_factor", "stall_checks")


def pair(inst, precision=0, **kw):
    """GPU handle and oracle LP of the same instance with the same PDHG parameters
    (no auxiliary columns: the LP relaxation exactly as given)."""
    S = lib()
    gp = S.default_params(precision=precision, aux_general_integers=0)
    op = O.PdhgParams()
    for k, v in kw.items():
        setattr(gp, k, int(v) if k != "fixed_step_factor" else float(v))
        if k in PDHG_KEYS:
            setattr(op, k, v)
    g = S.LP.from_instance(inst, gp)
    int_cols = np.nonzero(inst.is_int)[0]
    o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u, int_cols=int_cols, params=op)
    return g, o


def rel_err(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(1.0, float(np.max(np.abs(b)))))


def long_row_instance(seed=7, m=320, n=700):
    """Random LP with a few rows and columns longer than one warp tile (256 nnz) and
    empty rows, to cover the long-row path and ragged tiles."""
    rng = np.random.default_rng(seed)
    dense = np.where(rng.random((m, n)) < 0.01, rng.lognormal(size=(m, n)), 0.0)
    dense[3, :] = rng.uniform(0.5, 2.0, size=n)        # 700-nonzero rows
    dense[100, :] = rng.uniform(0.5, 2.0, size=n)
    dense[:, 11] = rng.uniform(0.5, 2.0, size=m)       # 320-nonzero columns
    dense[:, 500] = rng.uniform(0.5, 2.0, size=m)
    dense[7, :] = 0.0                                  # empty rows
    dense[250, :] = 0.0
    x0 = rng.uniform(1, 9, size=n)
    r = dense @ x0
    s = rng.uniform(0.05, 0.5, size=m)
    cov = rng.random(m) < 0.5
    lo = np.where(cov, r * (1 - s), -INF)
    hi = np.where(cov, INF, r * (1 + s))
    lo[7] = -1.0
    hi[250] = 1.0
    A = sp.csr_matrix(dense)
    A.sort_indices()
    c = rng.normal(size=n)
    return I.Instance("long_rows", m, n, A.indptr.astype(np.int64), A.indices.astype(np.int32),
                      A.data.astype(np.float64), c, lo, hi, np.zeros(n), np.full(n, 10.0),
                      (rng.random(n) < 0.3).astype(np.uint8))


def parity_instances():
    return {
        "setcover_200x500": I.set_cover(),
        "packcover_2kx4k": I.packing_covering(m=2000, n=4000, per_col=10, seed=11),
        "long_rows": long_row_instance(),
        "mcf_small": I.mcf(nodes=30, avg_degree=4, commodities=12, seed=5),
        "knapcover_700": I.knapsack_cover(700, seed=3),
    }


EPS = 2.0 ** -52
MARGIN = 1e-4  # relative closeness of a restart/candidate comparison that counts as a tie
LONG_MARGIN = 5e-2  # the same on long replays, whose states differ by up to TOL_LONG
# weighted KKT below which a long replay's residuals are the two trajectories'
# difference (states apart by TOL_LONG relative, entries O(1) after scaling) rather
# than the iterate's: one converged LP reached 9e-13 with the candidates' order flipped
LONG_KKT_FLOOR = 1e-8


def check_decisions(steps, checks, trace, replayed, long_run=False):
    """The oracle's own decisions, computed on the same trajectory, against the
    device's: step sizes within a tolerance scaled by the condition number of the
    interaction term, accept/restart/candidate choices equal unless the deciding
    quantities are within their rounding margins."""
    own_steps = [t for t in trace if t[0] == "step"]
    own_checks = [t for t in trace if t[0] == "check"]
    assert len(own_steps) == len(steps) and len(own_checks) == len(checks)
    for (_, k, acc, eta_used, eta_max, eta_next, cond, step_cond), rec in zip(own_steps, steps):
        if replayed:
            assert eta_used == rec[0]
        else:
            assert abs(eta_used - rec[0]) <= 1e-12 * eta_used
        # eta_max is a ratio of quadratic forms of the step: well conditioned when the
        # interaction term does not cancel (cond) and the step is not tiny against the
        # iterate (step_cond); otherwise only a sanity bound applies
        well = cond <= 1e6 and step_cond <= 1e4
        tol = 1e-6 if well else 1e-2
        if long_run:
            # after a few hundred attempts the replayed states differ in directions the
            # step sizes see (dy in non-unique dual directions), so the step-size values
            # are not compared; the accept decision still is, wherever the step is well
            # conditioned and the step size lies outside LONG_MARGIN of eta_max
            if well and np.isfinite(eta_max) and abs(eta_used - eta_max) > LONG_MARGIN * eta_max:
                assert acc == (rec[2] > 0.5), (k, eta_used, eta_max, rec)
            continue
        if np.isfinite(eta_max) and np.isfinite(rec[1]):
            assert abs(eta_max - rec[1]) <= tol * eta_max, (k, eta_max, rec[1], cond)
            assert abs(eta_next - rec[3]) <= tol * eta_next, (k, eta_next, rec[3], cond)
        else:
            assert np.isinf(eta_max) == np.isinf(rec[1]) or cond > 1e12
        tie = abs(eta_used - eta_max) <= tol * max(eta_max, 1e-300)
        assert tie or acc == (rec[2] > 0.5), (k, eta_used, eta_max, rec)
    for (_, k, restart, is_avg, omega_after, kc, rmargin, cmargin, wcond), rec in zip(own_checks, checks):
        assert k == rec[0]
        if long_run:
            # past convergence the weighted KKT values are rounding noise: the restart
            # and candidate decisions are compared where the candidate KKT is above
            # LONG_KKT_FLOOR, both sides measure it alike (within LONG_MARGIN), and it
            # lies outside LONG_MARGIN of every threshold and of the other candidate
            if kc > LONG_KKT_FLOOR and abs(kc - rec[4]) <= LONG_MARGIN * kc:
                assert rmargin <= LONG_MARGIN or restart == (rec[1] > 0.5), (k, restart, rmargin, rec)
                assert cmargin <= LONG_MARGIN or is_avg == (rec[2] > 0.5), (k, is_avg, cmargin, rec)
            continue
        assert abs(kc - rec[4]) <= MARGIN * kc, (k, kc, rec)
        assert rmargin <= MARGIN or restart == (rec[1] > 0.5), (k, restart, rec)
        assert cmargin <= MARGIN or is_avg == (rec[2] > 0.5), (k, is_avg, rec)
        if restart == (rec[1] > 0.5) and is_avg == (rec[2] > 0.5) and not long_run:
            assert abs(omega_after - rec[3]) <= (1e-9 + 1e-9 * wcond) * omega_after, (k, omega_after, rec, wcond)


def compare_after(inst, k, replay=True, tol=None, **kw):
    """k attempts of the device and of the oracle from the same cold start (the oracle
    on the device's decisions when replay is set): iterates, counts, step size and
    primal weight, and the decisions the oracle takes itself (check_decisions)."""
    tol = TOL if tol is None else tol
    g, o = pair(inst, trace_capacity=k + 8, **kw)
    rg = g.pdhg_solve(0.0, k)
    steps, checks = g.trace()
    assert len(steps) == k
    ro = o.solve(0.0, k, trace=True, replay=(steps, checks) if replay else None)
    xg, yg, eta_g, om_g = g.get_state()
    assert rg.status == ro.status == O.ITER_LIMIT
    assert rg.iterations == ro.iterations == k
    assert (rg.accepted, rg.rejected, rg.restarts) == (ro.accepted, ro.rejected, ro.restarts)
    ex = rel_err(xg, o.primal())
    ey = rel_err(yg, o.dual())
    if ey > tol:
        # y is not unique where it only reaches columns held at a bound (and modulo
        # the null space of A^T, e.g. the conservation rows of one commodity sum to
        # zero): the part of y the primal step sees is A^T y on the columns strictly
        # inside their bounds, so compare that
        A = inst.csr()
        xo = o.primal()
        free = (xo > inst.l + 1e-7 * (1 + np.abs(inst.l))) & (xo < inst.u - 1e-7 * (1 + np.abs(inst.u)))
        ey = min(ey, rel_err((A.T @ yg)[free], (A.T @ o.dual())[free]))
    assert ex <= tol and ey <= tol, (ex, ey)
    # which candidate is reported is a tie-break once both have converged to round-off
    assert bool(rg.used_average) == ro.used_average or max(rg.rel_kkt, ro.rel_kkt) < 1e-10
    check_decisions(steps, checks, ro.trace, replay, long_run=k > 100)
    assert abs(eta_g - o.eta) <= 1e-9 * o.eta and abs(om_g - o.omega) <= 1e-9 * o.omega
    assert abs(rg.rel_kkt - ro.rel_kkt) <= 1e-7 * max(1.0, ro.rel_kkt)
    g.close()
