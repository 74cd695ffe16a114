"""Continuous repair (the LP with the integer columns fixed at xhat, solved by the
same PDHG path) and the column-bound update it rests on, against the oracle.

- scylla_set_col_bounds + cold restart: fixed-step iterates equal the oracle's on
  the LP with the new bounds (FP64 within 1e-9; FP32-mixed within FP32 rounding).
- scylla_repair in fixed-step mode: the repaired point equals the oracle repair's
  within 1e-9, integer entries exactly xhat's.
- scylla_repair with the default adaptive rules: same verdict as the oracle, same
  objective within 1e-7, and the oracle's feasibility test agrees with the device's.
- An infeasible fixing is not found; malformed input is rejected.
- scylla_run with the repair finds the mixed packing/covering solutions the oracle's
  loop with the repair finds (round 1, found by the repair), each MIP-feasible.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg as O
from oracle import pump as P
from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import gpu_available, lib, pair, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

MIXED_TOL = 2e-5


def mixed_instance(seed, m=300, n=600):
    return I.packing_covering(m=m, n=n, per_col=4, seed=seed)


def fixed_bounds(inst, xhat):
    isi = inst.is_int == 1
    l = inst.l.copy()
    u = inst.u.copy()
    l[isi] = xhat[isi]
    u[isi] = xhat[isi]
    return l, u


@pytest.mark.parametrize("precision", [0, 1])
def test_set_col_bounds_then_fixed_step_matches_oracle(precision):
    inst = mixed_instance(31)
    l, u = fixed_bounds(inst, inst.meta["x0"])
    g, _ = pair(inst, precision=precision, adaptive_step=False, restarts=False)
    g.set_col_bounds(l, u)
    g.reset_state()
    k = 32 if precision == 0 else 1
    g.pdhg_solve(0.0, k)
    o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, l, u,
                   params=O.PdhgParams(adaptive_step=False, restarts=False))
    o.solve(0.0, k)
    x, y, _, _ = g.get_state()
    tol = 1e-9 if precision == 0 else MIXED_TOL
    assert rel_err(x, o.primal()) <= tol and rel_err(y, o.dual()) <= tol
    isi = inst.is_int == 1
    assert np.max(np.abs(g.primal()[isi] - inst.meta["x0"][isi])) <= 1e-6  # fixed columns stay put
    g.close()


def test_repair_fixed_step_matches_oracle_repair():
    inst = mixed_instance(32)
    xhat = inst.meta["x0"].copy()
    g, _ = pair(inst, adaptive_step=False, restarts=False)
    r, x = g.repair(xhat, 0.0, 64)
    st, xo, info = P.repair(inst, xhat, 0.0, 64, O.PdhgParams(adaptive_step=False, restarts=False))
    assert r.iterations == info["iterations"] == 64 and r.rounds == info["rounds"]
    assert rel_err(x, xo) <= 1e-9
    isi = inst.is_int == 1
    assert np.array_equal(x[isi], xhat[isi])
    assert r.status == st
    g.close()


@pytest.mark.parametrize("seed", [33, 34, 35])
def test_repair_converges_like_oracle(seed):
    inst = mixed_instance(seed)
    xhat = inst.meta["x0"].copy()
    g, _ = pair(inst)
    r, x = g.repair(xhat, 1e-9, 100000)
    st, xo, info = P.repair(inst, xhat, 1e-9, 100000)
    assert r.status == st == P.FOUND
    assert r.rel_kkt <= 1e-9
    assert abs(r.objective - float(inst.c @ xo)) <= 1e-7 * max(1.0, abs(r.objective))
    assert abs(r.objective - float(inst.c @ x)) <= 1e-9 * max(1.0, abs(r.objective))
    isi = inst.is_int == 1
    assert np.array_equal(x[isi], xhat[isi])
    assert P.check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u, inst.is_int, x)
    # the same LP from the mixed-precision handle: the repair copy solves in FP64
    gm, _ = pair(inst, precision=1)
    rm, xm = gm.repair(xhat, 1e-9, 100000)
    assert rm.status == P.FOUND and abs(rm.objective - r.objective) <= 1e-7 * max(1.0, abs(r.objective))
    g.close()
    gm.close()


def test_repair_infeasible_fixing_and_bad_input():
    S = lib()
    A = sp.csr_matrix(np.array([[1.0, 1.0], [1.0, 1.0]]))
    inst = I.Instance("fix", 2, 2, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data,
                      np.array([1.0, 1.0]), np.array([-math.inf, 0.5]), np.array([1.5, math.inf]),
                      np.zeros(2), np.array([3.0, 1.0]), np.array([1, 0], dtype=np.uint8))
    g = S.LP.from_instance(inst, S.default_params())
    r, x = g.repair(np.array([2.0, 0.0]), 1e-9, 20000)
    assert r.status == P.NOT_FOUND and x[0] == 2.0 and r.rounds == 0 and r.iterations == 0
    r, x = g.repair(np.array([1.0, 0.0]), 1e-9, 20000)
    assert r.status == P.FOUND and x[0] == 1.0 and abs(x[1]) <= 1e-7
    with pytest.raises(S.ScyllaError):
        g.repair(np.array([0.5, 0.0]), 1e-9, 100)  # fractional on the integer column
    with pytest.raises(S.ScyllaError):
        g.repair(np.array([4.0, 0.0]), 1e-9, 100)  # outside [0, 3]
    with pytest.raises(S.ScyllaError):
        g.set_col_bounds(np.array([1.0, 0.0]), np.array([0.0, 1.0]))  # lo > hi
    with pytest.raises(S.ScyllaError):
        g.set_col_bounds(np.array([0.5, 0.0]), np.array([1.0, 1.0]))  # fractional integer bound
    g.close()


def test_run_with_repair_finds_mixed_solutions():
    S = lib()
    for seed in range(300, 306):
        inst = I.packing_covering(m=40, n=80, per_col=4, seed=seed)
        g = S.LP.from_instance(inst, S.default_params(max_rounds=10, iter_limit=5000, repair_iters=20000))
        r, x = g.run()
        o = P.pump(inst, P.PumpParams(max_rounds=10, iter_limit=5000, repair_iters=20000))
        assert o.status == P.FOUND and o.found_by == "repair"
        assert r.status == 0 and r.found_by == 3 and r.rounds == 1
        assert P.check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u, inst.is_int, x)
        assert abs(r.objective - float(inst.c @ x)) <= 1e-9 * max(1.0, abs(r.objective))
        g.close()


@pytest.mark.parametrize("seed", range(3))
def test_pure_integer_run_with_repair_equals_run_without(seed):
    """Every column integer: the propagation screen ends each repair without a solve,
    so scylla_run with the repair gives the run without it, attempts included."""
    S = lib()
    inst = I.knapsack_cover(60, seed=900 + seed, per_col=4)
    out = []
    for rep in (0, 20000):
        g = S.LP.from_instance(inst, S.default_params(max_rounds=8, iter_limit=3000, repair_iters=rep))
        r, x = g.run()
        out.append((r.status, r.rounds, r.total_iterations, r.found_by, x.tobytes()))
        g.close()
    assert out[0] == out[1]
