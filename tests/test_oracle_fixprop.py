"""Pins of the fix-and-propagate oracle (Section 2.3) to hand-checkable rows and to
an independent fixpoint computation (CPU only)."""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fixprop as F
from paper_2307_03466_gb300 import instances as I

INF = math.inf


def csr(dense):
    A = sp.csr_matrix(np.array(dense, dtype=float))
    A.sort_indices()
    return A.indptr, A.indices, A.data


def test_cover_row_forces_last_variable():
    # x1 + x2 + x3 >= 1 with x1 = x2 = 0 fixed  =>  x3 >= 1
    rp, ci, v = csr([[1, 1, 1]])
    dl, du, ign = F.propagate_only(rp, ci, v, [1.0], [INF], [0, 0, 0], [0, 0, 1], [1, 1, 1])
    assert list(dl) == [0, 0, 1] and list(du) == [0, 0, 1] and not ign[0]


def test_knapsack_row_rounds_down():
    # 3 x1 + 5 x2 <= 7 with x2 = 1  =>  x1 <= floor(2/3) = 0
    rp, ci, v = csr([[3, 5]])
    dl, du, _ = F.propagate_only(rp, ci, v, [-INF], [7.0], [0, 1], [5, 1], [1, 1])
    assert du[0] == 0 and dl[0] == 0


def test_continuous_bound_is_not_rounded():
    # 3 x1 + 5 x2 <= 7, x2 = 1, x1 continuous in [0,5]  =>  x1 <= 2/3
    rp, ci, v = csr([[3, 5]])
    dl, du, _ = F.propagate_only(rp, ci, v, [-INF], [7.0], [0, 1], [5, 1], [0, 1])
    assert du[0] == (7.0 - 5.0) / 3.0


def test_infinite_contribution_does_not_tighten():
    # x1 + x2 <= 4 with x2 unbounded below: nothing can be said about x1
    rp, ci, v = csr([[1, 1]])
    dl, du, _ = F.propagate_only(rp, ci, v, [-INF], [4.0], [0, -INF], [10, 10], [1, 1])
    assert du[0] == 10
    # ... but x2 <= 4 - 0 = 4 is implied (only x2's own bound is infinite)
    assert du[1] == 4


def test_contradictory_rows_first_wins_second_ignored():
    # row0: x1 + x2 >= 2 ; row1: x1 + x2 <= 1 ; binaries
    rp, ci, v = csr([[1, 1], [1, 1]])
    dl, du, ign = F.propagate_only(rp, ci, v, [2.0, -INF], [INF, 1.0], [0, 0], [1, 1], [1, 1])
    assert list(dl) == [1, 1] and list(du) == [1, 1]
    assert not ign[0] and ign[1]


def test_small_slack_tolerance_is_integer_safe():
    # 2 x <= 2.0000001: floor(1.00000005 + 1e-6) = 1 ; 2 x >= 1.9999999: ceil(0.99999995 - 1e-6) = 1
    rp, ci, v = csr([[2.0]])
    dl, du, _ = F.propagate_only(rp, ci, v, [1.9999999], [2.0000001], [0], [5], [1])
    assert dl[0] == 1 and du[0] == 1


def sweep_fixpoint(rp, ci, v, lo, hi, l, u):
    """Independent greatest fixpoint: repeat full sweeps of the textbook interval rule
    (x_j in [(lo - maxact_{-j})/a, (hi - minact_{-j})/a], rounded inward) until nothing
    changes.  Integer data only, so every quantity is exact."""
    m = len(rp) - 1
    dl = [float(t) for t in l]
    du = [float(t) for t in u]
    changed = True
    while changed:
        changed = False
        for i in range(m):
            idx = range(rp[i], rp[i + 1])
            for p in idx:
                j, a = ci[p], v[p]
                others_min = sum(min(v[q] * dl[ci[q]], v[q] * du[ci[q]]) for q in idx if q != p)
                others_max = sum(max(v[q] * dl[ci[q]], v[q] * du[ci[q]]) for q in idx if q != p)
                lo_t = (lo[i] - others_max) if lo[i] > -INF else -INF
                hi_t = (hi[i] - others_min) if hi[i] < INF else INF
                if a > 0:
                    nl, nu = lo_t / a, hi_t / a
                else:
                    nl, nu = hi_t / a, lo_t / a
                nl = math.ceil(nl - 1e-6) if nl > -INF else -INF
                nu = math.floor(nu + 1e-6) if nu < INF else INF
                if nl > dl[j]:
                    dl[j] = float(nl); changed = True
                if nu < du[j]:
                    du[j] = float(nu); changed = True
                assert dl[j] <= du[j]
    return dl, du


@pytest.mark.parametrize("seed", range(25))
def test_queue_propagation_reaches_greatest_fixpoint(seed):
    """For feasible integer data the FIFO queue must land on the same domains as the
    order-free sweep (tightening is monotone, so the greatest fixpoint is unique)."""
    rng = np.random.default_rng(seed)
    m, n = 6, 7
    dense = np.where(rng.random((m, n)) < 0.5, rng.integers(-4, 5, size=(m, n)), 0)
    x0 = rng.integers(0, 6, size=n)
    r = dense @ x0
    lo = np.where(rng.random(m) < 0.5, r - rng.integers(0, 3, size=m), -INF).astype(float)
    hi = np.where(rng.random(m) < 0.5, r + rng.integers(0, 3, size=m), INF).astype(float)
    l = np.zeros(n); u = np.full(n, 8.0)
    rp, ci, v = csr(dense)
    dl, du, ign = F.propagate_only(rp, ci, v, lo, hi, l, u, np.ones(n))
    assert not ign.any()  # x0 is feasible, so no row can be contradictory
    sl, su = sweep_fixpoint(list(rp), list(ci), list(v), lo, hi, l, u)
    assert list(dl) == sl and list(du) == su
    assert np.all(dl <= x0) and np.all(x0 <= du)  # every feasible point survives


def brute_feasible(dense, lo, hi, x):
    a = dense @ x
    return bool(np.all(a >= lo - 1e-9) and np.all(a <= hi + 1e-9))


@pytest.mark.parametrize("seed", range(15))
def test_output_contract_on_small_binary_instances(seed):
    """Section 2.3: output integral on I and inside the final domains; domains shrink
    monotonically; with no ignored row, the rows were enforced by propagation so any
    violated row must have been ignored."""
    inst = I.set_cover(m=12, n=10, seed=seed, smin=1, smax=4)
    rng = np.random.default_rng(seed)
    xbar = rng.random(inst.n)
    xhat, dl, du, fixed, ign = F.fix_and_propagate(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi,
                                                   inst.l, inst.u, inst.is_int, xbar)
    assert np.all(xhat == np.floor(xhat))
    assert np.all(dl <= xhat) and np.all(xhat <= du)
    assert np.all(dl >= inst.l) and np.all(du <= inst.u)
    dense = inst.csr().toarray()
    if not ign.any():
        assert brute_feasible(dense, inst.lo, inst.hi, xhat)
    # set cover: propagation alone can always repair, so nothing is ignored
    assert not ign.any()


def test_fixing_order_most_integral_first():
    xbar = np.array([0.5, 0.9, 0.2, 0.1, 0.45, 2.0])
    order = F.fixing_order(xbar, [1, 1, 1, 1, 1, 0])
    # distances: 0.5, 0.1, 0.2, 0.1, 0.45 ; ties broken by index
    assert order == [1, 3, 2, 4, 0]


def test_infeasible_fix_is_ignored_and_still_integral():
    # x1 + x2 = 1 (equality) and x1 + x2 >= 2 are contradictory
    rp, ci, v = csr([[1, 1], [1, 1]])
    xhat, dl, du, fixed, ign = F.fix_and_propagate(rp, ci, v, [1.0, 2.0], [1.0, INF], [0, 0], [1, 1], [1, 1],
                                                   np.array([0.5, 0.5]))
    assert ign.any()
    assert set(xhat) <= {0.0, 1.0}


def test_unfixed_continuous_takes_projection():
    # x1 integer in [0,3], x2 continuous in [0,10]; x1 + x2 <= 4
    rp, ci, v = csr([[1, 1]])
    xhat, dl, du, fixed, ign = F.fix_and_propagate(rp, ci, v, [-INF], [4.0], [0, 0], [3, 10], [1, 0],
                                                   np.array([2.6, 9.0]))
    # x1 fixed to 3, then x2 <= 1, projection of 9 onto [0,1] is 1
    assert xhat[0] == 3 and xhat[1] == 1.0


def test_exhaustive_tiny_binary_soundness():
    """Whenever F&P's output satisfies the rows it is a true MIP solution: checked by
    enumerating all binary points of tiny instances."""
    for seed in range(30):
        rng = np.random.default_rng(1000 + seed)
        m, n = 3, 4
        dense = rng.integers(-2, 3, size=(m, n)).astype(float)
        lo = rng.integers(-2, 2, size=m).astype(float)
        hi = lo + rng.integers(0, 3, size=m)
        feas = [x for x in itertools.product([0, 1], repeat=n) if brute_feasible(dense, lo, hi, np.array(x, float))]
        rp, ci, v = csr(dense)
        xhat, _, _, _, ign = F.fix_and_propagate(rp, ci, v, lo, hi, np.zeros(n), np.ones(n), np.ones(n),
                                                 rng.random(n))
        if brute_feasible(dense, lo, hi, xhat):
            assert tuple(int(t) for t in xhat) in {tuple(f) for f in feas}
        if not feas:
            assert not brute_feasible(dense, lo, hi, xhat)


def test_visit_cap_stops_a_ping_pong_in_closed_form():
    """Rows x - y >= 1 and y - x >= 1 on integers in [0, U]: each visit moves one lower
    and one upper bound by one unit past the other column's, and the FIFO alternates
    the two rows, so visit k sets the bounds it touches to k and U - k.  With U = 1e9
    the domains would take 5e8 visits to cross; the call stops after
    visit_cap(2) = 20 * 2 + 1000 = 1040 visits with row 0's bounds from visit 1039
    and row 1's from visit 1040, and no row ignored."""
    U = 1e9
    assert F.visit_cap(2) == 1040
    dl, du, ign = F.propagate_only([0, 2, 4], [0, 1, 0, 1], [1.0, -1.0, -1.0, 1.0], [1.0, 1.0],
                                   [math.inf, math.inf], [0.0, 0.0], [U, U], [1, 1])
    assert list(dl) == [1039.0, 1040.0]
    assert list(du) == [U - 1040.0, U - 1039.0]
    assert not ign.any()
