"""Pins of the oracle's diagonal-QP mode (min c^T x + 1/2 x^T diag(q) x over the LP's
constraints; the primal step becomes the closed-form prox) and of the l2 pump
objective built on it.

- A box-only separable QP: x* = clip(-c/q, l, u) in closed form.
- One equality row, free columns: the Lagrange closed form.
- Tiny QPs with rows and boxes: brute force over active sets (every equality-
  constrained QP of a candidate active set, the feasible candidate of least
  objective is the unique minimizer of the strictly convex QP).
- q = 0 reproduces the LP iterates bit for bit.
- The l2 objective update: a hand example, and c_hat^T x + 1/2 x^T Q x + offset equals
  alpha^K s c^T x + (1 - alpha^K)/2 ||x_I - xhat_I||^2 at random points.
- The outer loop with the l2 distance returns only MIP-feasible points, and finds
  solutions with general integers without auxiliary columns.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg as O
from oracle import pump as P
from paper_2307_03466_gb300 import instances as I


def test_box_qp_closed_form():
    rng = np.random.default_rng(3)
    n = 12
    c = rng.normal(size=n)
    q = rng.uniform(0.5, 3.0, size=n)
    l = np.full(n, -0.4)
    u = np.full(n, 0.6)
    lp = O.OracleLP(sp.csr_matrix((0, n)), c, np.zeros(0), np.zeros(0), l, u, q=q)
    r = lp.solve(1e-12, 100000)
    assert r.status == O.CONVERGED
    np.testing.assert_allclose(lp.primal(), np.clip(-c / q, l, u), atol=1e-9)


def test_equality_qp_lagrange_closed_form():
    rng = np.random.default_rng(4)
    n = 8
    a = rng.uniform(0.5, 2.0, size=n)
    c = rng.normal(size=n)
    q = rng.uniform(0.5, 2.0, size=n)
    b = 3.0
    A = sp.csr_matrix(a.reshape(1, n))
    lp = O.OracleLP(A, c, np.array([b]), np.array([b]), np.full(n, -np.inf), np.full(n, np.inf), q=q)
    r = lp.solve(1e-11, 200000)
    assert r.status == O.CONVERGED
    lam = (b + np.sum(a * c / q)) / np.sum(a * a / q)
    x = (lam * a - c) / q
    np.testing.assert_allclose(lp.primal(), x, atol=1e-7)
    assert abs(r.pobj - (c @ x + 0.5 * np.sum(q * x * x))) <= 1e-8 * (1 + abs(r.pobj))


def brute_force_qp(dense, lo, hi, l, u, c, q):
    """Minimizer of c^T x + 1/2 sum q x^2 over lo <= Ax <= hi, l <= x <= u (q > 0)."""
    m, n = dense.shape
    cons = []  # (row vector, value) of every bound that can be active
    for i in range(m):
        opts = [None]
        if np.isfinite(lo[i]):
            opts.append((dense[i], lo[i]))
        if np.isfinite(hi[i]) and hi[i] != lo[i]:
            opts.append((dense[i], hi[i]))
        cons.append(opts)
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cons.append([None, (e, l[j]), (e, u[j])])
    best, best_f = None, math.inf
    Q = np.diag(q)
    for pick in itertools.product(*cons):
        act = [p for p in pick if p is not None]
        if len(act) > n:
            continue
        if act:
            G = np.array([g for g, _ in act])
            h = np.array([v for _, v in act])
            K = np.block([[Q, G.T], [G, np.zeros((len(act), len(act)))]])
            rhs = np.concatenate([-c, h])
        else:
            K, rhs = Q, -c
        try:
            sol = np.linalg.solve(K, rhs)
        except np.linalg.LinAlgError:
            continue
        x = sol[:n]
        ax = dense @ x
        tol = 1e-9
        if np.any(ax < lo - tol) or np.any(ax > hi + tol) or np.any(x < l - tol) or np.any(x > u + tol):
            continue
        f = c @ x + 0.5 * np.sum(q * x * x)
        if f < best_f:
            best, best_f = x, f
    return best, best_f


@pytest.mark.parametrize("seed", range(4))
def test_tiny_qp_matches_active_set_brute_force(seed):
    inst = I.tiny_lp(seed, m=3, n=4)
    dense = inst.meta["dense"]
    q = np.random.default_rng(seed + 50).uniform(0.3, 2.0, size=inst.n)
    lp = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u, q=q)
    r = lp.solve(1e-10, 400000)
    assert r.status == O.CONVERGED
    x, f = brute_force_qp(dense, inst.lo, inst.hi, inst.l, inst.u, inst.c, q)
    assert x is not None
    np.testing.assert_allclose(lp.primal(), x, atol=1e-6)
    assert abs(r.pobj - f) <= 1e-7 * (1 + abs(f))


def test_zero_hessian_is_the_lp_bit_for_bit():
    inst = I.tiny_lp(7, m=4, n=6)
    a = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
    b = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u, q=np.zeros(inst.n))
    ra = a.solve(0.0, 300)
    rb = b.solve(0.0, 300)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.y, b.y) and ra.pobj == rb.pobj


def test_l2_objective_update_hand_example():
    c = np.array([3.0, -4.0, 1.0])  # ||c|| = sqrt(26)
    is_int = np.array([1, 0, 1], dtype=np.uint8)
    xhat = np.array([2.0, 0.5, -1.0])
    chat, q, off = P.objective_update_l2(c, is_int, xhat, K=1, alpha=0.9)
    t = 0.9 * math.sqrt(2) / math.sqrt(26)
    om = 1.0 - 0.9  # 0.1 in binary floating point
    np.testing.assert_allclose(chat, [t * 3 - om * 2, t * -4, t * 1 + om * 1], rtol=1e-15)
    np.testing.assert_array_equal(q, [om, 0.0, om])
    assert abs(off - 0.5 * om * (4 + 1)) <= 1e-16


def test_l2_objective_equals_scaled_cost_plus_distance():
    rng = np.random.default_rng(9)
    n = 30
    c = rng.normal(size=n)
    is_int = (rng.random(n) < 0.5).astype(np.uint8)
    xhat = np.round(rng.uniform(-3, 3, size=n))
    for K in (1, 4, 20):
        chat, q, off = P.objective_update_l2(c, is_int, xhat, K)
        aK = 0.9 ** K
        s = math.sqrt(int(is_int.sum())) / float(np.linalg.norm(c))
        for _ in range(5):
            x = rng.uniform(-4, 4, size=n)
            lhs = chat @ x + 0.5 * np.sum(q * x * x) + off
            ii = is_int == 1
            rhs = aK * s * (c @ x) + (1 - aK) * 0.5 * np.sum((x[ii] - xhat[ii]) ** 2)
            assert abs(lhs - rhs) <= 1e-12 * (1 + abs(rhs))


@pytest.mark.parametrize("seed", range(3))
def test_l2_pump_is_sound_and_handles_general_integers(seed):
    inst = I.knapsack_cover(40, seed=500 + seed, per_col=4)
    inst_g = I.packing_covering(m=30, n=60, per_col=4, seed=600 + seed)  # general integers in [0, 10]
    for ins in (inst, inst_g):
        r = P.pump(ins, P.PumpParams(max_rounds=30, iter_limit=5000, distance=2))
        if r.status == P.FOUND:
            assert P.check_feasible(ins.rowptr, ins.cols, ins.vals, ins.lo, ins.hi, ins.l, ins.u, ins.is_int, r.x)
