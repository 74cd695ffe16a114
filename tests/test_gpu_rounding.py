"""The host rounding step and the objective update of the library against the oracle.

Fix-and-propagate fixings and domains must match bit for bit given the same
fractional point (Section 2.3); the feasibility test, the perturbation and the
objective update (Section 2.4) must agree with the oracle; every solution the
pump returns must pass an exact feasibility check.  These go through the C ABI,
whose handle lives on the GPU, hence the gpu mark.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fixprop as F
from oracle import pdhg as O
from oracle import pump as P
from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import gpu_available, lib, long_row_instance

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def handle(inst, **kw):
    S = lib()
    return S.LP.from_instance(inst, S.default_params(**kw))


ROUNDING_INSTANCES = {
    "setcover_200x500": lambda: I.set_cover(),
    "knapcover_300": lambda: I.knapsack_cover(300, seed=8),
    "packcover_gen_int": lambda: I.packing_covering(m=300, n=600, per_col=4, seed=21),
    "mcf_small": lambda: I.mcf(nodes=20, avg_degree=4, commodities=6, seed=2),
    "long_rows": lambda: long_row_instance(),
}


def xbar_points(inst, seed):
    rng = np.random.default_rng(seed)
    pts = [np.clip(rng.uniform(inst.l, np.minimum(inst.u, inst.l + 10)), inst.l, inst.u)]
    # an LP point from the oracle
    lp = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
    lp.solve(1e-3, 3000)
    pts.append(lp.primal())
    # exact halves exercise the round-half-up rule and the ordering ties
    h = np.floor(pts[0]) + 0.5
    pts.append(np.clip(h, inst.l, inst.u))
    return pts


@pytest.mark.parametrize("name", list(ROUNDING_INSTANCES))
def test_fix_and_propagate_bit_exact(name):
    inst = ROUNDING_INSTANCES[name]()
    g = handle(inst)
    for xb in xbar_points(inst, 5):
        xg, dlg, dug, fxg, igg = g.fix_and_propagate(xb)
        xo, dlo, duo, fxo, igo = F.fix_and_propagate(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi,
                                                    inst.l, inst.u, inst.is_int, xb)
        assert np.array_equal(xg, xo)
        assert np.array_equal(dlg, dlo) and np.array_equal(dug, duo)
        assert np.array_equal(fxg, fxo)
        assert np.array_equal(igg, igo)
        assert np.all(xg[inst.is_int == 1] == np.floor(xg[inst.is_int == 1]))
    g.close()


@pytest.mark.parametrize("name", ["setcover_200x500", "packcover_gen_int", "long_rows"])
def test_fix_and_propagate_many_points_bit_exact(name):
    """scylla_fix_and_propagate_many on the handle's host copies: every point as the
    oracle rounds it, and as a single call does."""
    inst = ROUNDING_INSTANCES[name]()
    g = handle(inst)
    pts = xbar_points(inst, 7)
    xh, nf = g.fix_and_propagate_many(np.stack(pts))
    for k, xb in enumerate(pts):
        xo, dlo, duo, fxo, igo = F.fix_and_propagate(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi,
                                                    inst.l, inst.u, inst.is_int, xb)
        assert np.array_equal(xh[k], xo) and nf[k] == len(fxo)
        assert np.array_equal(xh[k], g.fix_and_propagate(xb)[0])
    g.close()


def test_farkas_gap_on_a_device_handle():
    """scylla_farkas_gap through the binding, on a handle with auxiliary columns (its
    rows and columns are the original MIP's): D = 1 on an LP built infeasible, and
    the oracle's value on random multipliers of a feasible one."""
    from oracle import infeas as X
    from tests.test_oracle_infeas import _admissible_y
    inst = I.packing_covering(m=40, n=80, per_col=4, seed=100)
    rng = np.random.default_rng(0)
    A = inst.csr()
    ys = _admissible_y(inst, rng)
    L = X._side_min(ys, inst.lo, inst.hi)
    A2 = sp.vstack([A, sp.csr_matrix(A.T @ ys)]).tocsr()
    bad = I.Instance("built_infeasible", inst.m + 1, inst.n, A2.indptr.astype(np.int64),
                     A2.indices.astype(np.int32), A2.data, inst.c, np.append(inst.lo, -np.inf),
                     np.append(inst.hi, L - 1.0), inst.l, inst.u, inst.is_int)
    g = handle(bad)
    assert g.n_aux > 0
    assert abs(g.farkas_gap(np.append(ys, -1.0)) - 1.0) <= 1e-9 * (1.0 + abs(L))
    g.close()
    g = handle(inst)
    for _ in range(5):
        y = _admissible_y(inst, rng)
        go = X.farkas_gap(A, inst.lo, inst.hi, inst.l, inst.u, y)
        gl = g.farkas_gap(y)
        assert gl <= 1e-9 * (1.0 + abs(go)) and abs(gl - go) <= 1e-9 * (1.0 + abs(go))
    g.close()


@pytest.mark.parametrize("name", ["setcover_200x500", "knapcover_300", "packcover_gen_int"])
def test_feasibility_check_matches_oracle(name):
    inst = ROUNDING_INSTANCES[name]()
    g = handle(inst)
    rng = np.random.default_rng(1)
    pts = [np.ones(inst.n), np.zeros(inst.n)]
    for _ in range(20):
        x = rng.uniform(inst.l, np.minimum(inst.u, inst.l + 10))
        x[inst.is_int == 1] = np.round(x[inst.is_int == 1])
        pts.append(x)
    if "x0" in inst.meta:
        pts.append(inst.meta["x0"])
    for x in pts:
        assert g.check_feasible(x) == P.check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi,
                                                       inst.l, inst.u, inst.is_int, x)
    g.close()


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("K", [1, 2, 17])
def test_perturbation_matches_oracle(kind, K):
    inst = I.packing_covering(m=200, n=400, per_col=3, seed=4)
    g = handle(inst)
    rng = np.random.default_rng(K)
    xbar = rng.uniform(inst.l, np.minimum(inst.u, 10))
    xhat = xbar.copy()
    ic = np.nonzero(inst.is_int)[0]
    xhat[ic] = np.floor(xbar[ic] + 0.5)
    key = tuple(float(xhat[j]) for j in ic)
    other = tuple(v + 1 for v in key)
    hist = [key] if kind == 1 else [key, other]
    xo, _ = P.perturb(xhat, xbar, hist, K, 12345, list(ic), inst.l, inst.u)
    xg, nflip = g.perturb(xhat, xbar, kind, K, 12345)
    assert np.array_equal(xg, xo)
    assert nflip == int(np.sum(xg != xhat))
    g.close()


@pytest.mark.parametrize("K", [1, 3, 40])
def test_objective_update_matches_oracle(K):
    inst = I.packing_covering(m=100, n=300, per_col=3, seed=9)  # binaries are absent: general integers
    inst.is_int[:40] = 1
    inst.u[:20] = 1.0  # some binary-like integer columns
    g = handle(inst)
    rng = np.random.default_rng(K)
    xhat = rng.uniform(inst.l, inst.u)
    ic = inst.is_int == 1
    xhat[ic] = np.floor(xhat[ic] + 0.5)
    xhat[:5] = inst.l[:5]
    xhat[5:10] = inst.u[5:10]
    g.set_objective(xhat, K)
    chat, off = g.get_objective()
    gi = P.general_integer_columns(inst.is_int, inst.l, inst.u)
    assert g.n_aux == len(gi)
    co, aux_lo, offo = P.objective_update(inst.c, inst.is_int, inst.l, inst.u, xhat, K, gi)
    np.testing.assert_allclose(chat, co, rtol=1e-15, atol=1e-15)
    assert abs(off - offo) <= 1e-12 * (1 + abs(offo))
    g.close()


def test_objective_update_then_solve_matches_oracle_pump_lp():
    """The augmented LP after one objective update solves like the oracle's."""
    inst = I.packing_covering(m=150, n=300, per_col=3, seed=13)
    S = lib()
    g = S.LP.from_instance(inst, S.default_params(trace_capacity=600))
    A = inst.csr()
    aug = P.augment(A, inst.c, inst.lo, inst.hi, inst.l, inst.u, inst.is_int)
    o = O.OracleLP(aug.A, aug.c, aug.lo, aug.hi, aug.l, aug.u, int_cols=np.nonzero(inst.is_int)[0])
    rg = g.pdhg_solve(1e-2, 20000)
    ro = o.solve(1e-2, 20000)
    assert rg.iterations == ro.iterations
    xb = g.primal()
    xhat, *_ = g.fix_and_propagate(xb)
    g.set_objective(xhat, 1)
    chat, aux_lo, off = P.objective_update(inst.c, inst.is_int, inst.l, inst.u, xhat, 1, aug.gen_int)
    o.set_objective_vector(chat, off)
    lo2 = o.lo.copy()
    lo2[aug.m_orig:] = aux_lo
    o.set_row_bounds(lo2, o.hi)
    x, y, eta, om = g.get_state()
    o.set_state(x, y)
    o.eta, o.omega = eta, om
    rg = g.pdhg_solve(0.0, 500)
    ro = o.solve(0.0, 500, replay=g.trace())
    xg, yg, _, _ = g.get_state()
    from tests.gpu_common import rel_err
    assert rel_err(xg, o.primal()) <= 1e-9 and rel_err(yg, o.dual()) <= 1e-9
    g.close()


def brute_feasible(inst, x, tol=1e-9):
    a = inst.csr() @ x
    return bool(np.all(a >= inst.lo - tol) and np.all(a <= inst.hi + tol) and np.all(x >= inst.l)
                and np.all(x <= inst.u) and np.all(x[inst.is_int == 1] == np.round(x[inst.is_int == 1])))


def test_run_set_cover_finds_feasible_solution():
    inst = I.set_cover()
    g = handle(inst)
    r, x = g.run()
    assert r.status == 0
    assert brute_feasible(inst, x)
    assert P.check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u, inst.is_int, x)
    assert abs(r.objective - float(inst.c @ x)) < 1e-9
    g.close()


@pytest.mark.parametrize("seed", range(6))
def test_run_is_sound_on_knapsack_covers(seed):
    inst = I.knapsack_cover(60, seed=100 + seed, per_col=4)
    g = handle(inst, max_rounds=30, iter_limit=5000)
    r, x = g.run()
    if r.status == 0:
        assert brute_feasible(inst, x)
    g.close()


def test_run_reports_not_found_on_infeasible_instance():
    A = sp.csr_matrix(np.array([[1.0, 1.0]]))
    inst = I.Instance("infeasible", 1, 2, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data,
                      np.array([1.0, 1.0]), np.array([3.0]), np.array([np.inf]), np.zeros(2), np.ones(2),
                      np.ones(2, dtype=np.uint8))
    g = handle(inst, max_rounds=5, iter_limit=2000)
    r, _ = g.run()
    assert r.status == 1 and r.rounds == 5
    g.close()
