"""Pins of the oracle's continuous repair (the LP with the integer columns fixed
at xhat, solved by the oracle PDHG; the paper keeps the continuous part of the
fix-and-propagate point at the LP values, Section 2.3).

- The repaired objective equals the optimum of the same fixed LP from an
  independent solver (scipy's HiGHS), so a dropped fixing, a wrong bound or a
  wrong objective fails.
- The integer entries come back exactly as xhat's.
- A fixing that leaves the LP infeasible is reported as not found, by the
  propagation screen and without a solve.
- Where one solve leaves single rows violated beyond the check's tolerance, the
  shift rounds (violated rows' working bounds moved inward, warm re-solve) end
  at points that pass the exact check, near the fixed LP's optimum.
- In the outer loop the repair finds solutions of mixed packing/covering
  instances in round 1 that the loop without it misses, and every one passes the
  exact feasibility test.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

from oracle import pump as P
from paper_2307_03466_gb300 import instances as I


def fixed_lp_optimum(inst, xhat):
    """min c^T x over lo <= Ax <= hi, x_I = xhat_I, l <= x <= u elsewhere (HiGHS)."""
    A = sp.csr_matrix((inst.vals, inst.cols, inst.rowptr), shape=(inst.m, inst.n))
    isi = inst.is_int == 1
    l = inst.l.copy()
    u = inst.u.copy()
    l[isi] = xhat[isi]
    u[isi] = xhat[isi]
    fh, fl = np.isfinite(inst.hi), np.isfinite(inst.lo)
    Aub = sp.vstack([A[fh], -A[fl]]).tocsr()
    bub = np.concatenate([inst.hi[fh], -inst.lo[fl]])
    r = linprog(inst.c, A_ub=Aub, b_ub=bub, bounds=list(zip(l, u)), method="highs")
    return r


@pytest.mark.parametrize("seed", range(3))
def test_repair_objective_matches_highs(seed):
    inst = I.packing_covering(m=30, n=60, per_col=4, seed=200 + seed)
    xhat = inst.meta["x0"].copy()  # integral on the integer columns, feasible by construction
    st, x, info = P.repair(inst, xhat, 1e-9, 200000)
    ref = fixed_lp_optimum(inst, xhat)
    assert ref.status == 0 and st == P.FOUND
    assert abs(float(inst.c @ x) - ref.fun) <= 1e-7 * max(1.0, abs(ref.fun))


def test_repair_keeps_integer_entries_exact():
    inst = I.packing_covering(m=30, n=60, per_col=4, seed=201)
    xhat = inst.meta["x0"].copy()
    xhat[inst.is_int == 0] = 1e9  # continuous entries of xhat are ignored
    st, x, _ = P.repair(inst, xhat, 1e-9, 200000)
    isi = inst.is_int == 1
    assert st == P.FOUND
    assert np.array_equal(x[isi], inst.meta["x0"][isi])
    assert np.all(x[~isi] >= inst.l[~isi] - 1e-9) and np.all(x[~isi] <= inst.u[~isi] + 1e-9)


def test_repair_infeasible_fixing_is_not_found():
    # x0 integer in [0, 3], x1 continuous in [0, 1]: x0 + x1 <= 1.5 and x0 + x1 >= 0.5
    A = sp.csr_matrix(np.array([[1.0, 1.0], [1.0, 1.0]]))
    inst = I.Instance("fix", 2, 2, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data,
                      np.array([1.0, 1.0]), np.array([-math.inf, 0.5]), np.array([1.5, math.inf]),
                      np.zeros(2), np.array([3.0, 1.0]), np.array([1, 0], dtype=np.uint8))
    st, x, info = P.repair(inst, np.array([2.0, 0.0]), 1e-9, 20000)  # 2 + x1 <= 1.5 is impossible
    assert st == P.NOT_FOUND and x[0] == 2.0
    assert info["rounds"] == 0 and info["iterations"] == 0  # the propagation proves it, no solve runs
    st, x, _ = P.repair(inst, np.array([1.0, 0.0]), 1e-9, 20000)  # x1 = 0 works (objective 1)
    assert st == P.FOUND and x[0] == 1.0 and abs(x[1]) <= 1e-7


@pytest.mark.parametrize("seed", [201, 202, 205])
def test_shift_rounds_repair_points_one_solve_leaves_infeasible(seed):
    """At rel-KKT 1e-6 one solve leaves rows violated beyond the check's tolerance on
    these instances; moving the violated rows' working bounds inward and solving
    again gives points that pass the exact check, within a small gap of the fixed
    LP's optimum (HiGHS)."""
    inst = I.packing_covering(m=30, n=60, per_col=4, seed=seed)
    xhat = inst.meta["x0"]
    st1, _, info1 = P.repair(inst, xhat, 1e-6, 200000, rounds=1)
    st, x, info = P.repair(inst, xhat, 1e-6, 200000, rounds=8)
    assert st1 == P.NOT_FOUND and st == P.FOUND and info["rounds"] > 1 and info["shifted_rows"] > 0
    assert P.check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u, inst.is_int, x)
    ref = fixed_lp_optimum(inst, xhat)
    obj = float(inst.c @ x)
    assert obj >= ref.fun - 1e-5 * abs(ref.fun) and obj <= ref.fun + 1e-3 * abs(ref.fun)


def test_pump_with_repair_finds_mixed_solutions():
    found_off = found_on = 0
    for seed in range(300, 306):
        inst = I.packing_covering(m=40, n=80, per_col=4, seed=seed)
        r0 = P.pump(inst, P.PumpParams(max_rounds=10, iter_limit=5000))
        r1 = P.pump(inst, P.PumpParams(max_rounds=10, iter_limit=5000, repair_iters=20000))
        found_off += r0.status == P.FOUND
        found_on += r1.status == P.FOUND
        assert r1.status == P.FOUND and r1.found_by == "repair" and r1.rounds == 1
        assert P.check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u, inst.is_int,
                                r1.x)
    assert found_on == 6 and found_off < found_on


@pytest.mark.parametrize("seed", range(3))
def test_pure_integer_repairs_end_at_the_propagation_screen(seed):
    """With every column integer, a failed fixing leaves no continuous freedom: the
    screen proves each fixed LP infeasible, so the loop with the repair takes the
    same path, attempts included, as the loop without it."""
    inst = I.knapsack_cover(40, seed=900 + seed, per_col=4)
    r0 = P.pump(inst, P.PumpParams(max_rounds=8, iter_limit=3000))
    r1 = P.pump(inst, P.PumpParams(max_rounds=8, iter_limit=3000, repair_iters=20000))
    assert r0.status == r1.status and r0.rounds == r1.rounds and r0.total_iterations == r1.total_iterations
