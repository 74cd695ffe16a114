"""Pins of the infeasibility certificates (oracle/infeas.py) against hand examples,
weak duality on feasible LPs, and HiGHS's verdicts on LPs built to be infeasible or
unbounded."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

from oracle import infeas as X
from paper_2307_03466_gb300 import instances as I

INF = math.inf


def test_two_contradicting_rows():
    """x >= 1 and x <= 0 on a free x: y = (1, -1) aggregates them to 0 >= 1."""
    A = sp.csr_matrix(np.array([[1.0], [1.0]]))
    lo, hi, l, u = [1.0, -INF], [INF, 0.0], [-INF], [INF]
    assert X.farkas_gap(A, lo, hi, l, u, [1.0, -1.0]) == 1.0
    assert X.farkas_gap(A, lo, hi, l, u, [3.0, -3.0]) == 3.0  # D is positively homogeneous
    assert X.farkas_gap(A, lo, hi, l, u, [1.0, 0.0]) == -INF  # leans on x <= +inf
    assert X.farkas_gap(A, lo, hi, l, u, [-1.0, 1.0]) == -INF  # leans on the rows' infinite sides


def test_row_against_the_box():
    """x1 + x2 >= 3 over [0, 1]^2 cannot hold; >= 2 can, at the corner."""
    A = sp.csr_matrix(np.array([[1.0, 1.0]]))
    assert X.farkas_gap(A, [3.0], [INF], [0.0, 0.0], [1.0, 1.0], [1.0]) == 1.0
    assert X.farkas_gap(A, [2.0], [INF], [0.0, 0.0], [1.0, 1.0], [1.0]) == 0.0
    assert X.farkas_gap(A, [3.0], [INF], [0.0, 0.0], [1.0, 1.0], [-1.0]) == -INF


def test_unbounded_direction_by_hand():
    """min -x1 s.t. x1 - x2 <= 1, x >= 0: along d = (1, 1) the row stays put and the
    objective falls; d = (1, 0) leaves the row."""
    A = sp.csr_matrix(np.array([[1.0, -1.0]]))
    c, lo, hi, l, u = [-1.0, 0.0], [-INF], [1.0], [0.0, 0.0], [INF, INF]
    assert X.is_dual_ray(A, c, lo, hi, l, u, [1.0, 1.0])
    assert X.recession_violation(A, lo, hi, l, u, [1.0, 0.0]) == 1.0
    assert not X.is_dual_ray(A, c, lo, hi, l, u, [1.0, 0.0])
    assert not X.is_dual_ray(A, [1.0, 0.0], lo, hi, l, u, [1.0, 1.0])  # objective rises


def _admissible_y(inst, rng):
    """Random multipliers that use only finite row sides."""
    y = rng.normal(size=inst.m)
    y = np.where(np.isfinite(inst.lo), np.abs(y), 0.0) - np.where(np.isfinite(inst.hi), np.abs(rng.normal(size=inst.m)), 0.0)
    return y


@pytest.mark.parametrize("seed", range(5))
def test_weak_duality_on_feasible_lps(seed):
    """On an LP with a known feasible point no y certifies infeasibility: D(y) <= 0 up
    to the rounding of the sums, for every y tried."""
    inst = I.packing_covering(m=60, n=120, per_col=4, seed=seed)
    x0 = inst.meta["x0"]
    A = inst.csr()
    assert np.all(A @ x0 >= inst.lo - 1e-9) and np.all(A @ x0 <= inst.hi + 1e-9)
    rng = np.random.default_rng(seed)
    for _ in range(200):
        y = _admissible_y(inst, rng)
        g = X.farkas_gap(A, inst.lo, inst.hi, inst.l, inst.u, y)
        scale = float(np.abs(y) @ np.maximum(np.abs(np.nan_to_num(inst.lo, posinf=0, neginf=0)),
                                             np.abs(np.nan_to_num(inst.hi, posinf=0, neginf=0))))
        assert g <= 1e-9 * (1.0 + scale)


def _highs_status(A, c, lo, hi, l, u):
    A = sp.csr_matrix(A)
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    fh, fl = np.isfinite(hi), np.isfinite(lo)
    Aub = sp.vstack([A[fh], -A[fl]]).tocsr()
    bub = np.concatenate([hi[fh], -lo[fl]])
    r = linprog(c, A_ub=Aub, b_ub=bub, bounds=list(zip(l, u)), method="highs")
    return r.status  # 0 optimal, 2 infeasible, 3 unbounded


@pytest.mark.parametrize("seed", range(5))
def test_built_infeasible_lp_is_certified_and_highs_agrees(seed):
    """A feasible LP plus the row a^T x <= L - 1, where a = A^T y* and L is the least
    value the rows allow y*^T A x: the pair (y*, -1) certifies infeasibility with
    D = 1, while neither the new row alone nor y* alone does, and HiGHS reports the LP
    infeasible (and the original feasible)."""
    inst = I.packing_covering(m=40, n=80, per_col=4, seed=100 + seed)
    rng = np.random.default_rng(seed)
    A = inst.csr()
    ys = _admissible_y(inst, rng)
    a = A.T @ ys
    L = X._side_min(ys, inst.lo, inst.hi)
    assert math.isfinite(L)
    A2 = sp.vstack([A, sp.csr_matrix(a)]).tocsr()
    lo2 = np.append(inst.lo, -INF)
    hi2 = np.append(inst.hi, L - 1.0)
    y2 = np.append(ys, -1.0)
    g = X.farkas_gap(A2, lo2, hi2, inst.l, inst.u, y2)
    assert abs(g - 1.0) <= 1e-9 * (1.0 + abs(L))
    assert X.farkas_gap(A2, lo2, hi2, inst.l, inst.u, np.append(np.zeros(inst.m), -1.0)) <= 0.0
    assert X.farkas_gap(A, inst.lo, inst.hi, inst.l, inst.u, ys) <= 1e-9 * (1.0 + abs(L))
    assert _highs_status(A, inst.c, inst.lo, inst.hi, inst.l, inst.u) == 0
    assert _highs_status(A2, inst.c, lo2, hi2, inst.l, inst.u) == 2


def test_built_unbounded_lp_has_a_ray_and_highs_agrees():
    """A free column that no row touches, with a negative cost, makes the LP unbounded:
    e_j is a dual ray, and HiGHS says unbounded."""
    inst = I.packing_covering(m=30, n=60, per_col=3, seed=7)
    A = sp.hstack([inst.csr(), sp.csr_matrix((inst.m, 1))]).tocsr()
    c = np.append(inst.c, -1.0)
    l = np.append(inst.l, -INF)
    u = np.append(inst.u, INF)
    d = np.zeros(inst.n + 1)
    d[-1] = -1.0  # raises the objective: no ray
    assert not X.is_dual_ray(A, c, inst.lo, inst.hi, l, u, d)
    d[-1] = 1.0  # lowers it without bound
    assert X.is_dual_ray(A, c, inst.lo, inst.hi, l, u, d)
    assert _highs_status(A, c, inst.lo, inst.hi, l, u) == 3


def test_planted_sign_mistake_fails_the_built_certificate():
    """The rows' bound taken from the wrong side (hi for y > 0) turns the built
    certificate's D = 1 into something else."""
    def wrong_side_min(y, lo, hi):
        return X._side_min(y, hi, lo)
    inst = I.packing_covering(m=40, n=80, per_col=4, seed=100)
    rng = np.random.default_rng(0)
    A = inst.csr()
    ys = _admissible_y(inst, rng)
    a = A.T @ ys
    L = X._side_min(ys, inst.lo, inst.hi)
    A2 = sp.vstack([A, sp.csr_matrix(a)]).tocsr()
    lo2, hi2 = np.append(inst.lo, -INF), np.append(inst.hi, L - 1.0)
    y2 = np.append(ys, -1.0)
    right = X._box_max(A2.T @ y2, inst.l, inst.u)
    assert abs((X._side_min(y2, lo2, hi2) - right) - 1.0) <= 1e-9 * (1.0 + abs(L))
    assert not abs((wrong_side_min(y2, lo2, hi2) - right) - 1.0) <= 1e-9 * (1.0 + abs(L))


def _built_infeasible(seed, m=40, n=80):
    inst = I.packing_covering(m=m, n=n, per_col=4, seed=100 + seed)
    rng = np.random.default_rng(seed)
    A = inst.csr()
    ys = _admissible_y(inst, rng)
    L = X._side_min(ys, inst.lo, inst.hi)
    A2 = sp.vstack([A, sp.csr_matrix(A.T @ ys)]).tocsr()
    return inst, A2, np.append(inst.lo, -INF), np.append(inst.hi, L - 1.0)


@pytest.mark.parametrize("seed", range(8))
def test_detector_certifies_built_infeasible_lps(seed):
    """With infeasibility checks on, the default adaptive solve of each built infeasible
    LP ends INFEASIBLE within a few thousand attempts, with a ray that the independent
    test confirms (D > 0), on an LP that HiGHS reports infeasible."""
    from oracle import pdhg as O
    inst, A2, lo2, hi2 = _built_infeasible(seed, *((40, 80) if seed < 6 else (120, 240)))
    lp = O.OracleLP(A2, inst.c, lo2, hi2, inst.l, inst.u, params=O.PdhgParams(infeasibility_checks=True))
    r = lp.solve(1e-8, 5000)
    assert r.status == O.INFEASIBLE
    assert X.farkas_gap(A2, lo2, hi2, inst.l, inst.u, r.certificate) > 0
    assert _highs_status(A2, inst.c, lo2, hi2, inst.l, inst.u) == 2


def test_detector_certifies_a_row_against_its_box():
    from oracle import pdhg as O
    A = sp.csr_matrix(np.array([[1.0, 1.0], [1.0, -1.0]]))
    lo, hi = np.array([3.0, -1.0]), np.array([INF, 1.0])
    lp = O.OracleLP(A, np.array([1.0, 2.0]), lo, hi, np.zeros(2), np.ones(2),
                    params=O.PdhgParams(infeasibility_checks=True))
    r = lp.solve(1e-8, 5000)
    assert r.status == O.INFEASIBLE
    assert X.farkas_gap(A, lo, hi, np.zeros(2), np.ones(2), r.certificate) > 0


@pytest.mark.parametrize("name", ["setcover", "packcover", "knapcover", "mcf"])
def test_detector_never_fires_on_feasible_lps_and_changes_nothing(name):
    """On feasible LPs the checks cannot fire (weak duality; the margin is far above
    the rounding) and leave the trajectory bit for bit as it is without them."""
    from oracle import pdhg as O
    inst = {"setcover": lambda: I.set_cover(m=60, n=150, seed=3),
            "packcover": lambda: I.packing_covering(m=80, n=160, per_col=4, seed=5),
            "knapcover": lambda: I.knapsack_cover(80, seed=2),
            "mcf": lambda: I.mcf(nodes=12, avg_degree=4, commodities=4, seed=1)}[name]()
    res = []
    for on in (False, True):
        lp = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u,
                        params=O.PdhgParams(infeasibility_checks=on))
        r = lp.solve(1e-7, 6000)
        res.append((r.status, r.iterations, lp.primal().copy(), lp.dual().copy()))
    assert res[1][0] != O.INFEASIBLE
    assert res[0][:2] == res[1][:2]
    assert np.array_equal(res[0][2], res[1][2]) and np.array_equal(res[0][3], res[1][3])
