"""Pins of the outer-loop oracle (Algorithm 1, Sections 2.2-2.4) on CPU."""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pump as P
from oracle.pdhg import OracleLP
from paper_2307_03466_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
INF = math.inf


def test_tolerance_schedule_closed_form():
    # Section 2.2: eps^(1) = 0.01, eps^(K+1) = max(0.98 eps^(K), 1e-8)
    for K in (1, 2, 3, 10, 100, 684, 685, 686, 1000):
        closed = max(0.01 * 0.98 ** (K - 1), 1e-8)
        assert abs(P.eps_schedule(K) - closed) <= 1e-12 * closed
    # the floor is first reached at K = 1 + ceil(ln(1e-6) / ln(0.98)) = 685
    assert P.eps_schedule(684) > 1e-8 and P.eps_schedule(685) == 1e-8


def test_splitmix64_published_outputs():
    # SplitMix64 reference outputs for seed 0 (Steele, Lea, Flood 2014 generator)
    r = P.SplitMix64(0)
    assert [r.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    r = P.SplitMix64(0)
    u = [r.uniform() for _ in range(1000)]
    assert all(0.0 <= t < 1.0 for t in u)


def test_objective_update_hand_example():
    g = json.load(open(os.path.join(GOLDEN, "objective_update_example.json")))
    chat, aux_lo, off = P.objective_update(np.array(g["c"]), g["is_int"], g["l"], g["u"], g["xhat"], g["K"], [])
    np.testing.assert_allclose(chat, g["c_hat"], rtol=1e-14, atol=1e-15)
    assert abs(off - g["offset"]) < 1e-15
    assert len(aux_lo) == 0


def test_objective_update_distance_term_is_l1_distance():
    """For binaries, c_hat^T x + offset with alpha^K -> 0 equals the l1 distance to xhat."""
    rng = np.random.default_rng(0)
    n = 20
    c = rng.normal(size=n)
    is_int = (rng.random(n) < 0.6).astype(np.uint8)
    l = np.zeros(n); u = np.ones(n)
    xhat = np.where(is_int == 1, rng.integers(0, 2, size=n), 0.3)
    chat, _, off = P.objective_update(c, is_int, l, u, xhat, 400, [])  # 0.9^400 ~ 5e-19
    for _ in range(10):
        x = rng.random(n)
        d = sum(abs(x[j] - xhat[j]) for j in range(n) if is_int[j])
        assert abs(chat @ x + off - d) < 1e-12


def test_objective_update_zero_c():
    chat, _, off = P.objective_update(np.zeros(3), [1, 1, 0], [0, 0, 0], [1, 1, 1], [1.0, 0.0, 0.5], 1, [])
    np.testing.assert_allclose(chat, [-0.1, 0.1, 0.0], atol=1e-16)
    assert abs(off - 0.1) < 1e-16


def test_aux_rows_model_l1_distance_on_general_integers():
    """min d s.t. d - x >= -xhat, d + x >= xhat  equals |x - xhat| (Section 4 remark)."""
    A = sp.csr_matrix(np.array([[1.0]]))
    aug = P.augment(A, [0.0], [-INF], [INF], [0.0], [10.0], [1])
    assert aug.gen_int == [0] and aug.A.shape == (3, 2)
    for xh in (0.0, 3.0, 7.0, 10.0):
        chat, aux_lo, off = P.objective_update(np.array([0.0]), [1], [0.0], [10.0], [xh], 200, aug.gen_int)
        lo = aug.lo.copy(); lo[1:] = aux_lo
        for xv in (0.0, 2.5, 3.0, 9.0):
            # fix x by its bounds and solve the LP: optimum is |xv - xh|
            lp = OracleLP(aug.A, chat, lo, aug.hi, [xv, 0.0], [xv, 10.0])
            res = lp.solve(1e-10, 100000)
            assert abs(res.pobj - abs(xv - xh)) < 1e-6


def test_perturb_short_cycle_flips_largest_distances():
    n = 40
    xbar = np.linspace(0.01, 0.49, n)
    xhat = np.zeros(n)
    hist = [tuple(xhat)]
    x, kind = P.perturb(xhat, xbar, hist, 3, 7, list(range(n)), np.zeros(n), np.ones(n))
    assert kind == "short"
    r = P.SplitMix64(7 ^ 3)
    TT = 10 + int(math.floor(r.uniform() * 21))
    flipped = np.nonzero(x != xhat)[0]
    assert len(flipped) == TT
    assert set(flipped) == set(range(n - TT, n))  # the largest |xbar - xhat|


def test_perturb_long_cycle_hand_example():
    """A long cycle worked by hand (tests/golden/long_cycle_example.json): the
    uniforms of the round's stream are written out, and the flips follow from them
    column by column, binaries and general integers, with a continuous column
    between them that draws no uniform."""
    g = json.load(open(os.path.join(GOLDEN, "long_cycle_example.json")))
    r = P.SplitMix64(g["seed"] ^ g["K"])
    assert [r.uniform() for _ in g["uniforms_of_stream_seed_14"]] == g["uniforms_of_stream_seed_14"]
    hist = [tuple(float(v) for v in h) for h in g["history_int_keys"]]
    x, kind = P.perturb(np.array(g["xhat"], float), np.array(g["xbar"], float), hist, g["K"], g["seed"],
                        g["int_cols"], np.array(g["l"], float), np.array(g["u"], float))
    assert kind == g["expected_kind"]
    np.testing.assert_array_equal(x, np.array(g["expected_xhat"], float))


def test_perturb_no_cycle():
    n = 30
    xbar = np.random.default_rng(1).random(n)
    b = tuple(np.ones(n))
    x, kind = P.perturb(np.full(n, 0.0), xbar, [b], 5, 11, list(range(n)), np.zeros(n), np.ones(n))
    assert kind == "none"
    x, kind = P.perturb(np.full(n, 0.0), xbar, [], 5, 11, list(range(n)), np.zeros(n), np.ones(n))
    assert kind == "none"


def test_flip_general_integer():
    assert P._flip(3.0, 3.4, 0.0, 10.0) == 2.0  # at round(xbar): move away
    assert P._flip(3.0, 4.6, 0.0, 10.0) == 4.0  # toward xbar
    assert P._flip(0.0, 0.3, 0.0, 10.0) == 1.0  # away blocked by bound: other way
    assert P._flip(1.0, 0.2, 0.0, 1.0) == 0.0


def brute_feasible(inst, x, tol=1e-9):
    a = inst.csr() @ x
    return (np.all(a >= inst.lo - tol) and np.all(a <= inst.hi + tol) and np.all(x >= inst.l - tol)
            and np.all(x <= inst.u + tol) and np.all(x[inst.is_int == 1] == np.round(x[inst.is_int == 1])))


@pytest.mark.parametrize("seed", range(12))
def test_check_feasible_agrees_with_enumeration(seed):
    inst = I.knapsack_cover(6, seed=seed, per_col=3)
    for x in itertools.product([0.0, 1.0], repeat=inst.n):
        x = np.array(x)
        assert P.check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u,
                                inst.is_int, x) == brute_feasible(inst, x)


def test_check_feasible_tolerance_on_continuous_rows():
    rp, ci, v = np.array([0, 2]), np.array([0, 1]), np.array([0.1, 0.2])
    # 0.1 x0 + 0.2 x1 >= 0.3 at x = (1, 1): 0.30000000000000004 in FP64, passes
    assert P.check_feasible(rp, ci, v, [0.3], [INF], [0, 0], [1, 1], [0, 0], np.array([1.0, 1.0]))
    assert not P.check_feasible(rp, ci, v, [0.31], [INF], [0, 0], [1, 1], [0, 0], np.array([1.0, 1.0]))
    # integrality is exact
    assert not P.check_feasible(rp, ci, v, [0.0], [INF], [0, 0], [1, 1], [1, 0], np.array([0.5, 1.0]))


def test_pump_finds_set_cover_solution():
    inst = I.set_cover(m=40, n=80, seed=12)
    res = P.pump(inst, P.PumpParams(max_rounds=30))
    assert res.status == P.FOUND
    assert brute_feasible(inst, res.x)


@pytest.mark.parametrize("seed", range(4))
def test_pump_soundness_on_enumerable_instances(seed):
    inst = I.knapsack_cover(5, seed=200 + seed, per_col=3)
    feas = [x for x in itertools.product([0.0, 1.0], repeat=inst.n) if brute_feasible(inst, np.array(x))]
    res = P.pump(inst, P.PumpParams(max_rounds=15, iter_limit=5000))
    if res.status == P.FOUND:
        assert tuple(res.x) in set(feas)
    if not feas:
        assert res.status == P.NOT_FOUND


def test_pump_reports_not_found_on_infeasible_instance():
    # x0 + x1 >= 3 with binaries is infeasible
    A = sp.csr_matrix(np.array([[1.0, 1.0]]))
    inst = I.Instance("infeasible", 1, 2, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data,
                      np.array([1.0, 1.0]), np.array([3.0]), np.array([INF]), np.zeros(2), np.ones(2),
                      np.ones(2, dtype=np.uint8))
    res = P.pump(inst, P.PumpParams(max_rounds=5, iter_limit=2000))
    assert res.status == P.NOT_FOUND


def test_pump_with_general_integers_is_sound():
    inst = I.packing_covering(m=30, n=60, per_col=3, seed=5)
    res = P.pump(inst, P.PumpParams(max_rounds=10, iter_limit=4000))
    if res.status == P.FOUND:
        assert P.check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u,
                                inst.is_int, res.x)
