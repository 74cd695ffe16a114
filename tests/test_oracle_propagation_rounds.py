"""Pins of the oracle's round-based (Jacobi) propagation, the form the GPU runs.

- On integer data with a feasible point it reaches the independent greatest
  fixpoint (full sweeps of the textbook interval rule) and the FIFO propagation's
  domains bit for bit, with no row ignored and no conflict.
- A chain of k implications needs k + 1 rounds (closed form), and a hand example
  tightens as computed by hand.
- On mixed data every feasible point survives (soundness), whatever the order
  effects of the continuous thresholds.
"""
import numpy as np
import pytest

from oracle import fixprop as F
from tests.test_oracle_fixprop import csr, sweep_fixpoint

INF = np.inf


def integer_instance(seed, m=6, n=7):
    rng = np.random.default_rng(seed)
    dense = np.where(rng.random((m, n)) < 0.5, rng.integers(-4, 5, size=(m, n)), 0)
    x0 = rng.integers(0, 6, size=n)
    r = dense @ x0
    lo = np.where(rng.random(m) < 0.5, r - rng.integers(0, 3, size=m), -INF).astype(float)
    hi = np.where(rng.random(m) < 0.5, r + rng.integers(0, 3, size=m), INF).astype(float)
    return dense, x0, lo, hi, np.zeros(n), np.full(n, 8.0)


@pytest.mark.parametrize("seed", range(25))
def test_rounds_reach_the_fifo_and_sweep_fixpoint_on_integer_data(seed):
    dense, x0, lo, hi, l, u = integer_instance(seed)
    rp, ci, v = csr(dense)
    n = dense.shape[1]
    dl, du, ign, rounds, conflicts = F.propagate_rounds(rp, ci, v, lo, hi, l, u, np.ones(n))
    assert not ign.any() and conflicts == 0
    fl, fu, fign = F.propagate_only(rp, ci, v, lo, hi, l, u, np.ones(n))
    assert np.array_equal(dl, fl) and np.array_equal(du, fu)
    sl, su = sweep_fixpoint(list(rp), list(ci), list(v), lo, hi, l, u)
    assert list(dl) == sl and list(du) == su
    assert np.all(dl <= x0) and np.all(x0 <= du)


def test_chain_needs_one_round_per_link():
    # x_{k+1} >= x_k + 1 for k = 0..K-1 (rows -x_k + x_{k+1} >= 1), x_0 >= 2, x in [0, 20]
    K = 6
    n = K + 1
    dense = np.zeros((K + 1, n))
    for k in range(K):
        dense[k, k] = -1.0
        dense[k, k + 1] = 1.0
    dense[K, 0] = 1.0
    lo = np.array([1.0] * K + [2.0])
    hi = np.full(K + 1, INF)
    rp, ci, v = csr(dense)
    dl, du, ign, rounds, conflicts = F.propagate_rounds(rp, ci, v, lo, hi, np.zeros(n), np.full(n, 20.0), np.ones(n))
    np.testing.assert_array_equal(dl, 2.0 + np.arange(n))
    # round 1 sets x_0 >= 2 and x_1 >= 1 (from x_0 >= 0), ...; each further round moves the
    # front one link; the upper bounds tighten backwards from x_K <= 20 the same way
    assert rounds == K + 2 and conflicts == 0 and not ign.any()


def test_hand_example():
    # x + y <= 3 (integers in [0, 5]), x >= 2: round 1 gives x in [2, 3], y in [0, 3];
    # round 2 gives y in [0, 1]; round 3 changes nothing
    dense = np.array([[1.0, 1.0], [1.0, 0.0]])
    rp, ci, v = csr(dense)
    dl, du, ign, rounds, conflicts = F.propagate_rounds(rp, ci, v, np.array([-INF, 2.0]), np.array([3.0, INF]),
                                                        np.zeros(2), np.full(2, 5.0), np.ones(2))
    assert list(dl) == [2.0, 0.0] and list(du) == [3.0, 1.0] and rounds == 3


@pytest.mark.parametrize("seed", range(10))
def test_rounds_are_sound_on_mixed_data(seed):
    rng = np.random.default_rng(100 + seed)
    m, n = 8, 10
    dense = np.where(rng.random((m, n)) < 0.4, rng.normal(size=(m, n)), 0.0)
    is_int = (rng.random(n) < 0.5).astype(np.uint8)
    x0 = np.where(is_int == 1, rng.integers(0, 5, size=n), rng.uniform(0, 5, size=n)).astype(float)
    r = dense @ x0
    lo = np.where(rng.random(m) < 0.5, r - rng.uniform(0, 1, size=m), -INF)
    hi = np.where(rng.random(m) < 0.5, r + rng.uniform(0, 1, size=m), INF)
    rp, ci, v = csr(dense)
    dl, du, ign, rounds, conflicts = F.propagate_rounds(rp, ci, v, lo, hi, np.zeros(n), np.full(n, 6.0), is_int)
    assert not ign.any() and conflicts == 0
    assert np.all(dl <= x0 + 1e-9) and np.all(x0 <= du + 1e-9)
