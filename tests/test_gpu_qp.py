"""Diagonal quadratic objectives (scylla_set_qp_objective) and the l2-distance
objective update (distance = 2) against the oracle's diagonal-Hessian PDHG.

- Fixed-step iterates with a Hessian equal the oracle's: FP64 within 1e-9 in the
  32-row, wide and staged forms and the persistent kernel; FP32-mixed within FP32
  rounding.
- An all-zero Hessian leaves the LP path bit for bit.
- Adaptive solves reach rel-KKT 1e-8 (FP64) and 1e-4 (FP32-mixed) as the oracle's
  KKT evaluation of the returned point confirms, at the active-set optimum on tiny
  QPs.
- The l2 update: c_hat and the offset equal the oracle's, and the next fixed-step
  solve equals the oracle's with the same objective and Hessian.
- scylla_run with distance 2 returns only MIP-feasible points, with general
  integers and no auxiliary columns.
"""
import numpy as np
import pytest

from oracle import pdhg as O
from oracle import pump as P
from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import gpu_available, lib, long_row_instance, pair, rel_err
from tests.test_oracle_qp import brute_force_qp

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

MIXED_TOL = 2e-5


def hessian(inst, seed, frac=0.6):
    rng = np.random.default_rng(seed)
    return np.where(rng.random(inst.n) < frac, rng.uniform(0.1, 3.0, size=inst.n), 0.0)


def oracle_qp(inst, q, **kw):
    op = O.PdhgParams(**kw)
    return O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u, params=op, q=q)


@pytest.mark.parametrize("name,prefetch,mode", [("long_rows", 4, 1), ("long_rows", 2, 1), ("long_rows", 3, 1),
                                                ("packcover", 4, 1), ("packcover", 4, 3)])
def test_fixed_step_qp_iterates_match_oracle(name, prefetch, mode):
    inst = long_row_instance() if name == "long_rows" else I.packing_covering(m=300, n=600, per_col=4, seed=41)
    q = hessian(inst, 1)
    g, _ = pair(inst, adaptive_step=False, restarts=False, prefetch=prefetch, use_graph=mode)
    g.set_qp_objective(inst.c, q, 0.0)
    g.reset_state()
    g.pdhg_solve(0.0, 32)
    o = oracle_qp(inst, q, adaptive_step=False, restarts=False)
    o.solve(0.0, 32)
    x, y, _, _ = g.get_state()
    assert rel_err(x, o.primal()) <= 1e-9 and rel_err(y, o.dual()) <= 1e-9
    g.close()


def test_fixed_step_qp_mixed_one_attempt():
    inst = I.packing_covering(m=300, n=600, per_col=4, seed=42)
    q = hessian(inst, 2)
    g, _ = pair(inst, precision=1, adaptive_step=False, restarts=False)
    g.set_qp_objective(inst.c, q, 0.0)
    g.reset_state()
    g.pdhg_solve(0.0, 1)
    o = oracle_qp(inst, q, adaptive_step=False, restarts=False)
    o.solve(0.0, 1)
    x, y, _, _ = g.get_state()
    assert rel_err(x, o.primal()) <= MIXED_TOL and rel_err(y, o.dual()) <= MIXED_TOL
    g.close()


def test_zero_hessian_keeps_the_lp_path():
    inst = long_row_instance()
    a, _ = pair(inst)
    b, _ = pair(inst)
    b.set_qp_objective(inst.c, np.zeros(inst.n), 0.0)
    ra = a.pdhg_solve(1e-6, 5000)
    rb = b.pdhg_solve(1e-6, 5000)
    assert ra.iterations == rb.iterations
    assert np.array_equal(a.get_state()[0], b.get_state()[0]) and np.array_equal(a.get_state()[1], b.get_state()[1])
    a.close()
    b.close()


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-4)])
def test_adaptive_qp_converges_checked_by_oracle(precision, tol):
    inst = I.packing_covering(m=300, n=600, per_col=4, seed=43)
    q = hessian(inst, 3)
    g, _ = pair(inst, precision=precision)
    g.set_qp_objective(inst.c, q, 0.0)
    g.reset_state()
    r = g.pdhg_solve(tol, 200000)
    assert r.status == O.CONVERGED and r.rel_kkt <= tol
    o = oracle_qp(inst, q)
    x, y, _, _ = g.get_state()
    ev = o.evaluate(x / o.C, y / o.R)
    assert ev.rel_kkt <= 1.2 * tol, ev
    assert abs(ev.pobj - r.pobj) <= 1e-6 * (1 + abs(ev.pobj))
    g.close()


@pytest.mark.parametrize("seed", range(3))
def test_tiny_qp_reaches_active_set_optimum(seed):
    inst = I.tiny_lp(seed, m=3, n=4)
    q = np.random.default_rng(seed + 50).uniform(0.3, 2.0, size=inst.n)
    g, _ = pair(inst)
    g.set_qp_objective(inst.c, q, 0.0)
    g.reset_state()
    r = g.pdhg_solve(1e-10, 400000)
    x, f = brute_force_qp(inst.meta["dense"], inst.lo, inst.hi, inst.l, inst.u, inst.c, q)
    assert r.status == O.CONVERGED
    np.testing.assert_allclose(g.primal(), x, atol=1e-6)
    assert abs(r.pobj - f) <= 1e-7 * (1 + abs(f))
    g.close()


@pytest.mark.parametrize("K", [1, 5])
def test_l2_objective_update_matches_oracle(K):
    S = lib()
    inst = I.packing_covering(m=300, n=600, per_col=4, seed=44)  # general integers in [0, 10]
    g = S.LP.from_instance(inst, S.default_params(distance=2, adaptive_step=0, restarts=0))
    assert g.n_aux == 0
    g.pdhg_solve(1e-3, 2000)
    xhat = np.where(inst.is_int == 1, np.clip(np.round(g.primal()), inst.l, inst.u), 0.0)
    g.set_objective(xhat, K)
    chat, off = g.get_objective()
    oc, oq, ooff = P.objective_update_l2(inst.c, inst.is_int, xhat, K)
    np.testing.assert_allclose(chat, oc, rtol=0, atol=1e-15 * max(1.0, np.max(np.abs(oc))))
    assert abs(off - ooff) <= 1e-12 * max(1.0, abs(ooff))
    # the next solve with that objective and Hessian, from the same state
    x0, y0, eta, om = g.get_state()
    g.pdhg_solve(0.0, 16)
    o = O.OracleLP(inst.csr(), oc, inst.lo, inst.hi, inst.l, inst.u, offset=ooff, q=oq,
                   params=O.PdhgParams(adaptive_step=False, restarts=False))
    o.set_state(x0, y0)
    o.eta, o.omega = eta, om
    o.solve(0.0, 16)
    x, y, _, _ = g.get_state()
    assert rel_err(x, o.primal()) <= 1e-9 and rel_err(y, o.dual()) <= 1e-9
    g.close()


@pytest.mark.parametrize("seed", range(3))
def test_l2_run_is_sound(seed):
    S = lib()
    for inst in (I.knapsack_cover(60, seed=700 + seed, per_col=4),
                 I.packing_covering(m=40, n=80, per_col=4, seed=800 + seed)):
        g = S.LP.from_instance(inst, S.default_params(distance=2, max_rounds=30, iter_limit=5000))
        r, x = g.run()
        if r.status == 0:
            assert P.check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u,
                                    inst.is_int, x)
            assert abs(r.objective - float(inst.c @ x)) <= 1e-9 * max(1.0, abs(r.objective))
        g.close()
