"""Pins of the PDHG oracle to facts outside itself (CPU only).

Each test checks the oracle against something the paper or the mathematics fixes:
hand-computed steps of Algorithm 1, an independent LP solver (HiGHS via SciPy),
brute-force vertex enumeration, closed-form LPs, the fixed-point and
nonexpansiveness properties of PDHG, and strong duality.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

from oracle import pdhg as O
from paper_2307_03466_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = math.inf


def raw_params(**kw):
    """No preconditioning, so the oracle iterates the LP as given."""
    d = dict(ruiz_iters=0, pock_chambolle=False)
    d.update(kw)
    return O.PdhgParams(**d)


def highs(A, c, lo, hi, l, u):
    """Optimal primal/dual pair from HiGHS, in the oracle's sign convention
    (y_i >= 0 on an active lower row bound, <= 0 on an active upper one)."""
    A = sp.csr_matrix(A)
    m, n = A.shape
    eq = np.isfinite(lo) & np.isfinite(hi) & (lo == hi)
    ub_rows, ub_b, sgn, idx = [], [], [], []
    for i in range(m):
        if eq[i]:
            continue
        if np.isfinite(hi[i]):
            ub_rows.append(A[i].toarray().ravel()); ub_b.append(hi[i]); sgn.append(1.0); idx.append(i)
        if np.isfinite(lo[i]):
            ub_rows.append(-A[i].toarray().ravel()); ub_b.append(-lo[i]); sgn.append(-1.0); idx.append(i)
    eq_idx = np.nonzero(eq)[0]
    res = linprog(c, A_ub=np.array(ub_rows) if ub_rows else None, b_ub=np.array(ub_b) if ub_b else None,
                  A_eq=A[eq_idx].toarray() if len(eq_idx) else None, b_eq=lo[eq_idx] if len(eq_idx) else None,
                  bounds=list(zip(np.where(np.isfinite(l), l, None), np.where(np.isfinite(u), u, None))),
                  method="highs")
    assert res.status == 0, res.message
    y = np.zeros(m)
    if ub_rows:
        for k, i in enumerate(idx):
            # d obj / d(hi) = marginal; d obj / d(lo) = -marginal of the negated row
            y[i] += res.ineqlin.marginals[k] * (1.0 if sgn[k] > 0 else -1.0)
    if len(eq_idx):
        y[eq_idx] = res.eqlin.marginals
    return res.x, y, res.fun


def vertex_enumeration(dense, c, lo, hi, l, u):
    """Minimum of c^T x over the vertices of a small bounded polyhedron."""
    m, n = dense.shape
    G, h = [], []  # G x <= h
    for i in range(m):
        if np.isfinite(hi[i]):
            G.append(dense[i]); h.append(hi[i])
        if np.isfinite(lo[i]):
            G.append(-dense[i]); h.append(-lo[i])
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        G.append(e); h.append(u[j])
        G.append(-e); h.append(-l[j])
    G = np.array(G); h = np.array(h)
    best = INF
    for act in itertools.combinations(range(len(h)), n):
        M = G[list(act)]
        if abs(np.linalg.det(M)) < 1e-9:
            continue
        x = np.linalg.solve(M, h[list(act)])
        if np.all(G @ x <= h + 1e-9):
            best = min(best, float(c @ x))
    return best


def lp_of(inst, params=None):
    return O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u, params=params)


def test_two_by_two_hand_steps():
    g = json.load(open(os.path.join(GOLDEN, "pdhg_two_by_two.json")))
    A = sp.csr_matrix(np.array(g["A"]))
    lp = O.OracleLP(A, g["c"], g["b"], [INF, INF], g["l"], g["u"], params=raw_params())
    np.testing.assert_array_equal(lp.R, [1, 1])
    x = np.array(g["x0"]); y = np.array(g["y0"])
    eta = math.sqrt(g["tau_x"] * g["tau_y"]); omega = math.sqrt(g["tau_y"] / g["tau_x"])
    for st in g["steps"]:
        x, y = lp.pdhg_step(x, y, eta, omega)
        np.testing.assert_array_equal(x, st["x"])  # exact in binary floating point
        np.testing.assert_array_equal(y, st["y"])


def test_dual_step_reduces_to_paper_formula():
    rng = np.random.default_rng(5)
    y = rng.normal(size=1000)
    Axt = rng.normal(size=1000)
    b = rng.normal(size=1000)
    sigma = 0.37
    got = O.dual_prox(y, sigma, Axt, b, np.full(1000, INF))
    np.testing.assert_array_equal(got, np.maximum(0.0, y + sigma * (b - Axt)))
    # equality rows: no projection at all
    got = O.dual_prox(y, sigma, Axt, b, b)
    np.testing.assert_array_equal(got, y + sigma * (b - Axt))
    # <= rows: the mirror image, y' = min(0, ...)
    got = O.dual_prox(y, sigma, Axt, np.full(1000, -INF), b)
    np.testing.assert_array_equal(got, np.minimum(0.0, y + sigma * (b - Axt)))
    # free rows: y' = 0
    got = O.dual_prox(y, sigma, Axt, np.full(1000, -INF), np.full(1000, INF))
    np.testing.assert_array_equal(got, 0.0)


def test_dual_step_is_prox_of_row_support_function():
    """y' maximises lo*y^+ - hi*y^- - (y - v)^2 / (2 sigma), v = y - sigma*Axt, by grid search."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        lo, hi = sorted(rng.normal(size=2) * 3)
        if rng.random() < 0.3:
            lo = -INF
        if rng.random() < 0.3:
            hi = INF
        y, axt, sigma = rng.normal(), rng.normal() * 3, rng.uniform(0.1, 2)
        v = y - sigma * axt
        grid = np.linspace(-20, 20, 400001)
        with np.errstate(invalid="ignore"):
            f = (np.where(grid > 0, lo * np.maximum(grid, 0), 0.0) - np.where(grid < 0, hi * np.maximum(-grid, 0), 0.0)
                 - (grid - v) ** 2 / (2 * sigma))
        f = np.where(np.isnan(f), -INF, f)
        best = grid[np.argmax(f)]
        got = O.dual_prox(np.array([y]), sigma, np.array([axt]), np.array([lo]), np.array([hi]))[0]
        assert abs(got - best) < 2e-4


@pytest.mark.parametrize("seed", range(6))
def test_converges_to_vertex_enumeration_optimum(seed):
    inst = I.tiny_lp(seed, m=4, n=4)
    best = vertex_enumeration(inst.meta["dense"], inst.c, inst.lo, inst.hi, inst.l, inst.u)
    lp = lp_of(inst)
    res = lp.solve(1e-9, 200000)
    assert res.status == O.CONVERGED
    assert abs(res.pobj - best) <= 1e-6 * (1 + abs(best))


@pytest.mark.parametrize("seed", range(4))
def test_matches_highs_on_random_lps(seed):
    inst = I.tiny_lp(100 + seed, m=12, n=18, density=0.4)
    _, _, fstar = highs(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
    for params in (O.PdhgParams(), raw_params()):
        lp = lp_of(inst, params)
        res = lp.solve(1e-8, 400000)
        assert res.status == O.CONVERGED
        assert abs(res.pobj - fstar) <= 1e-5 * (1 + abs(fstar))
        assert abs(res.dobj - fstar) <= 1e-5 * (1 + abs(fstar))


def test_set_cover_relaxation_matches_highs():
    inst = I.set_cover(m=60, n=150, seed=3)
    _, _, fstar = highs(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
    lp = lp_of(inst)
    res = lp.solve(1e-7, 200000)
    assert res.status == O.CONVERGED
    assert abs(res.pobj - fstar) <= 1e-4 * (1 + abs(fstar))


def test_optimal_pair_is_fixed_point_and_has_zero_kkt():
    inst = I.tiny_lp(21, m=10, n=14, density=0.5)
    x, y, fstar = highs(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
    lp = lp_of(inst, raw_params())
    ev = lp.evaluate(x, y)
    assert ev.rel_kkt < 1e-7
    assert abs(ev.pobj - fstar) < 1e-7 * (1 + abs(fstar))
    assert abs(ev.dobj - fstar) < 1e-7 * (1 + abs(fstar))
    x1, y1 = lp.pdhg_step(x, y, 0.3, 1.0)
    assert np.max(np.abs(x1 - x)) < 1e-7
    assert np.max(np.abs(y1 - y)) < 1e-7
    # a perturbed point is not optimal
    ev2 = lp.evaluate(x + 0.1, y)
    assert ev2.rel_kkt > 1e-4


def test_kkt_is_invariant_under_preconditioning():
    inst = I.tiny_lp(33, m=15, n=20, density=0.4)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 4, size=inst.n)
    y = rng.normal(size=inst.m)
    y = np.where(np.isfinite(inst.lo), y, np.minimum(y, 0))
    y = np.where(np.isfinite(inst.hi), y, np.maximum(y, 0))
    a = lp_of(inst, raw_params())
    b = lp_of(inst, O.PdhgParams())
    assert not np.allclose(b.R, 1.0)
    ea = a.evaluate(x / a.C, y / a.R)
    eb = b.evaluate(x / b.C, y / b.R)
    for f in ("eps_p", "eps_d", "eps_g", "pobj", "dobj"):
        assert abs(getattr(ea, f) - getattr(eb, f)) <= 1e-12 * (1 + abs(getattr(ea, f)))


def test_box_lp_closed_form():
    rng = np.random.default_rng(2)
    n = 50
    c = rng.normal(size=n)
    l = rng.uniform(-5, 0, size=n)
    u = rng.uniform(0, 5, size=n)
    lp = O.OracleLP(sp.csr_matrix((0, n)), c, np.zeros(0), np.zeros(0), l, u)
    res = lp.solve(1e-10, 100000)
    assert res.status == O.CONVERGED
    np.testing.assert_allclose(lp.primal(), np.where(c > 0, l, u), atol=1e-8)


def test_fractional_knapsack_closed_form():
    rng = np.random.default_rng(4)
    n = 30
    a = rng.uniform(0.5, 3.0, size=n)
    c = rng.uniform(0.5, 3.0, size=n)
    u = np.ones(n)
    b = 0.4 * a.sum()
    # greedy by cost per unit of coverage
    order = np.argsort(c / a)
    need, f = b, 0.0
    for j in order:
        take = min(1.0, need / a[j])
        f += take * c[j]
        need -= take * a[j]
        if need <= 0:
            break
    lp = O.OracleLP(sp.csr_matrix(a[None, :]), c, [b], [INF], np.zeros(n), u)
    res = lp.solve(1e-10, 200000)
    assert res.status == O.CONVERGED
    assert abs(res.pobj - f) < 1e-7 * (1 + f)


def test_identity_matrix_closed_form():
    # min c^T x, lo <= x <= hi (rows), 0 <= x <= 10 (columns): separable
    rng = np.random.default_rng(8)
    n = 40
    c = rng.normal(size=n)
    lo = rng.uniform(1, 3, size=n)
    hi = lo + rng.uniform(0.5, 2, size=n)
    lp = O.OracleLP(sp.identity(n, format="csr"), c, lo, hi, np.zeros(n), np.full(n, 10.0))
    res = lp.solve(1e-10, 100000)
    assert res.status == O.CONVERGED
    np.testing.assert_allclose(lp.primal(), np.where(c > 0, lo, hi), atol=1e-7)


def test_fixed_step_pdhg_is_nonexpansive_in_M_norm():
    inst = I.tiny_lp(55, m=10, n=12, density=0.5)
    xs, ys, _ = highs(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
    lp = lp_of(inst, raw_params(adaptive_step=False, restarts=False))
    A = inst.csr().toarray()
    eta, omega = lp.eta, lp.omega
    tau, sigma = eta / omega, eta * omega
    assert tau * sigma * np.linalg.norm(A, 2) ** 2 < 1

    def mnorm(x, y):
        dx, dy = x - xs, y - ys
        return dx @ dx / tau + dy @ dy / sigma + 2 * dy @ (A @ dx)

    x = np.zeros(inst.n); y = np.zeros(inst.m)
    prev = mnorm(x, y)
    for _ in range(300):
        x, y = lp.pdhg_step(x, y, eta, omega)
        cur = mnorm(x, y)
        assert cur <= prev * (1 + 1e-12) + 1e-12
        prev = cur


def test_fixed_step_mode_makes_no_decisions():
    inst = I.tiny_lp(60, m=8, n=10)
    lp = lp_of(inst, O.PdhgParams(adaptive_step=False, restarts=False))
    res = lp.solve(0.0, 500, trace=True)
    assert res.status == O.ITER_LIMIT and res.rejected == 0 and res.restarts == 0
    assert all(t[2] for t in res.trace if t[0] == "step")


def test_adaptive_solve_takes_restarts_and_reports_iterations():
    inst = I.set_cover(m=40, n=100, seed=9)
    lp = lp_of(inst)
    res = lp.solve(1e-6, 100000, trace=True)
    assert res.status == O.CONVERGED
    assert res.iterations == res.accepted + res.rejected
    assert res.restarts >= 1


def test_iteration_limit_and_check_schedule():
    inst = I.tiny_lp(61, m=8, n=10)
    lp = lp_of(inst)
    res = lp.solve(0.0, 100)
    assert res.status == O.ITER_LIMIT and res.iterations == 100
    lp2 = lp_of(inst)
    res0 = lp2.solve(0.0, 0)
    assert res0.iterations == 0 and res0.status == O.ITER_LIMIT


def test_warm_start_keeps_state():
    inst = I.tiny_lp(62, m=8, n=10)
    lp = lp_of(inst)
    lp.solve(1e-8, 100000)
    x = lp.primal().copy()
    res = lp.solve(1e-8, 100000)
    assert res.iterations == 0  # already optimal: stops at the first check
    np.testing.assert_array_equal(lp.primal(), x)


def test_rounding_hash_is_order_independent_and_sensitive():
    cols = np.arange(100)
    x = np.random.default_rng(3).uniform(0, 5, size=100)
    h = O.rounding_hash(x, cols)
    perm = np.random.default_rng(4).permutation(100)
    assert O.rounding_hash(x[perm], cols[perm]) == h
    x2 = x.copy(); x2[17] = np.floor(x2[17] + 0.5) + 1.0
    assert O.rounding_hash(x2, cols) != h


# --- the relative KKT error at a point that is not optimal (Section 2.2) -------
def _golden_eval_lp(params):
    d = json.load(open(os.path.join(GOLDEN, "evaluate_nonoptimal.json")))
    f = lambda v: [float(t) for t in v]
    A = sp.csr_matrix(np.array(d["A_dense"], float))
    lp = O.OracleLP(A, f(d["c"]), f(d["row_lo"]), f(d["row_hi"]), f(d["col_lo"]), f(d["col_hi"]), params=params)
    return d, lp, np.array(f(d["x"])), np.array(f(d["y"]))


def test_evaluate_hand_example_at_a_nonoptimal_point():
    """Hand-computed eps_p, eps_d, eps_g, p and d (tests/golden/evaluate_nonoptimal.json)
    on an LP with covering, packing and two-sided rows and boxed, lower-only,
    upper-only and free columns: pins the normalisations 1 + ||b||, 1 + ||c||,
    1 + |p| + |d|, every branch of the reduced-cost projection and every bound
    term of the dual objective away from the optimum."""
    d, lp, x, y = _golden_eval_lp(raw_params())
    ev = lp.evaluate(x, y)
    e = d["expected"]
    assert abs(ev.eps_p - math.sqrt(7.5) / (1 + math.sqrt(19))) <= 1e-15
    assert abs(ev.eps_d - math.sqrt(11) / (1 + math.sqrt(32))) <= 1e-15
    assert abs(ev.eps_g - 6.75 / 10.25) <= 1e-15
    assert ev.pobj == e["pobj"] and ev.dobj == e["dobj"]
    for k in ("eps_p", "eps_d", "eps_g"):
        assert abs(getattr(ev, k) - e[k + "_value"]) <= 1e-15, k
    assert ev.rel_kkt == max(ev.eps_p, ev.eps_d, ev.eps_g)
    # with an objective offset of 1/2 both objectives move: 8.5, 1.75, eps_g = 0.6
    lp.set_objective_vector(lp.c, 0.5)
    ev = lp.evaluate(x, y)
    assert ev.pobj == 8.5 and ev.dobj == 1.75 and abs(ev.eps_g - 0.6) <= 1e-15


def test_evaluate_hand_example_through_the_preconditioned_lp():
    """The same point given to the preconditioned LP (x / C, y / R): the residuals
    are measured on the original LP, so the hand values stand."""
    d, lp, x, y = _golden_eval_lp(O.PdhgParams())
    assert not np.allclose(lp.R, 1.0) and not np.allclose(lp.C, 1.0)
    lp.set_state(x, y)
    ev = lp.evaluate(lp.x, lp.y)
    e = d["expected"]
    for k in ("eps_p", "eps_d", "eps_g"):
        assert abs(getattr(ev, k) - e[k + "_value"]) <= 1e-14, k
    assert abs(ev.pobj - 8.0) <= 1e-14 and abs(ev.dobj - 1.25) <= 1e-14


@pytest.mark.parametrize("gen,seed", [("open", 0), ("open", 1), ("open", 2), ("std", 0), ("std", 1)])
def test_open_bound_and_standard_form_lps_match_highs(gen, seed):
    """LPs with one-sided, free and fixed columns (and standard-form LPs: x >= 0,
    equality rows) built around a known optimal pair: HiGHS finds the constructed
    optimum, and the oracle's PDHG converges to it with its relative KKT error
    confirmed; the start proj_[l,u](0) has a nonzero dual residual, so the
    Lambda = R+, R- and {0} branches carry weight on the way."""
    inst = (I.open_bounds_lp(30, 60, seed=seed) if gen == "open" else I.standard_form_lp(30, 60, seed=seed))
    assert np.isinf(inst.u).any()
    if gen == "open":
        assert np.isinf(inst.l).any() and (np.isinf(inst.l) & np.isinf(inst.u)).any()
    _, _, fstar = highs(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
    assert abs(fstar - inst.meta["f_star"]) <= 1e-9 * (1 + abs(fstar))
    lp = lp_of(inst)
    ev0 = lp.evaluate(lp.x, lp.y)
    assert ev0.eps_d > 1e-3
    np.testing.assert_allclose(lp.primal(), np.clip(np.zeros(inst.n), inst.l, inst.u), rtol=1e-15, atol=0)
    res = lp.solve(1e-8, 400000)
    assert res.status == O.CONVERGED
    assert abs(res.pobj - fstar) <= 1e-6 * (1 + abs(fstar))
    assert abs(res.dobj - fstar) <= 1e-6 * (1 + abs(fstar))
    # the constructed pair itself has zero KKT error
    ev = lp_of(inst, raw_params()).evaluate(inst.meta["x_star"], inst.meta["y_star"])
    assert ev.rel_kkt <= 1e-13


def _planted_projection(mistake):
    def proj(r, l, u):
        lf, uf = np.isfinite(l), np.isfinite(u)
        if mistake == "cones_swapped":
            return np.where(lf & uf, r, np.where(lf, np.minimum(r, 0.0), np.where(uf, np.maximum(r, 0.0), 0.0)))
        # "one_sided_as_boxed": Lambda = R whenever one bound is finite
        return np.where(lf | uf, r, 0.0)
    return proj


def _planted_bound_norm(mistake):
    def bn(lo, hi):
        a = np.where(np.isfinite(lo), np.abs(lo), 0.0)
        b = np.where(np.isfinite(hi), np.abs(hi), 0.0)
        return a + b if mistake == "sum" else np.minimum(a, b)
    return bn


@pytest.mark.parametrize("mistake", ["cones_swapped", "one_sided_as_boxed", "sum", "min"])
def test_evaluate_hand_example_rejects_planted_mistakes(monkeypatch, mistake):
    """A wrong sign cone for one-sided columns, or a wrong bound norm, fails the
    hand example."""
    if mistake in ("cones_swapped", "one_sided_as_boxed"):
        monkeypatch.setattr(O, "reduced_cost_projection", _planted_projection(mistake))
    else:
        monkeypatch.setattr(O, "bound_norm_vector", _planted_bound_norm(mistake))
    with pytest.raises(AssertionError):
        test_evaluate_hand_example_at_a_nonoptimal_point()
