"""The seeded input generators produce the workloads as their recipe states them
(sizes, structure, value ranges, feasibility of the generating point, seeds)."""
import numpy as np
import pytest
from scipy.optimize import linprog
import scipy.sparse as sp

from paper_2307_03466_gb300 import instances as I


def _cols_rows(inst):
    return sp.csr_matrix((inst.vals, inst.cols, inst.rowptr), shape=(inst.m, inst.n)).tocsc()


def test_packing_covering_bench_workload_recipe():
    inst = I.packing_covering()
    assert (inst.m, inst.n, inst.nnz) == (50_000, 100_000, 1_000_000)
    At = _cols_rows(inst)
    assert np.all(np.diff(At.indptr) == 10)  # 10 nonzeros per column, at distinct rows
    assert np.all(inst.vals > 0)
    assert abs(inst.is_int.mean() - 0.30) < 0.01
    ic = inst.is_int == 1
    assert np.all(inst.l == 0) and np.all(inst.u[ic] == 10) and np.all(inst.u[~ic] == 100)
    # each row covering or packing (one finite side), the generating point inside by
    # a slack s in [0.05, 0.5] of its activity
    fin_lo, fin_hi = np.isfinite(inst.lo), np.isfinite(inst.hi)
    assert np.all(fin_lo ^ fin_hi)
    r = inst.csr() @ inst.meta["x0"]
    s = np.where(fin_lo, 1.0 - inst.lo / r, inst.hi / r - 1.0)
    assert np.all(s >= 0.05 - 1e-12) and np.all(s <= 0.5 + 1e-12)
    assert abs(fin_lo.mean() - 0.5) < 0.01
    x0 = inst.meta["x0"]
    assert np.all(x0[ic] == np.round(x0[ic])) and np.all((x0 >= inst.l) & (x0 <= inst.u))


def test_generators_are_reproducible_from_their_seeds():
    a, b = I.packing_covering(m=300, n=600, seed=5), I.packing_covering(m=300, n=600, seed=5)
    c = I.packing_covering(m=300, n=600, seed=6)
    for k in ("rowptr", "cols", "vals", "c", "lo", "hi", "l", "u", "is_int"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
    assert not np.array_equal(a.vals, c.vals)
    assert np.array_equal(I.set_cover().cols, I.set_cover().cols)


def test_set_cover_recipe():
    inst = I.set_cover()
    assert (inst.m, inst.n) == (200, 500)
    assert np.all(np.diff(inst.rowptr) >= 1)  # every row covered
    sizes = np.diff(_cols_rows(inst).indptr)
    assert sizes.min() >= 3 and np.mean(sizes) <= 8.5
    assert np.all((inst.c >= 1) & (inst.c <= 100) & (inst.c == np.round(inst.c)))
    assert np.all(inst.is_int == 1) and np.all(inst.lo == 1) and np.all(np.isinf(inst.hi))


def test_knapsack_cover_recipe():
    inst = I.knapsack_cover(400, seed=3)
    assert inst.n == 2 * inst.m
    assert np.all(np.diff(_cols_rows(inst).indptr) == 8)
    assert np.all((inst.vals >= 1) & (inst.vals <= 20) & (inst.vals == np.round(inst.vals)))
    assert np.all(np.isfinite(inst.lo) ^ np.isfinite(inst.hi))
    fin = np.concatenate([inst.lo[np.isfinite(inst.lo)], inst.hi[np.isfinite(inst.hi)]])
    assert np.all(fin == np.round(fin))
    assert np.all(inst.c != 0) and np.all(np.abs(inst.c) <= 10)


def test_power_law_sizes_follow_m_to_the_minus_two():
    """The CDF of p(m) ~ m^-2 on [a, b] is (1/a - 1/m) / (1/a - 1/b); the drawn sizes
    follow it (Kolmogorov distance below 0.02 on 20k draws)."""
    a, b = 1000, 50_000
    m = np.sort(I.power_law_sizes(20_000, a, b, seed=9)).astype(float)
    assert m.min() >= a and m.max() <= b
    F = (1 / a - 1 / m) / (1 / a - 1 / b)
    emp = np.arange(1, len(m) + 1) / len(m)
    assert np.max(np.abs(emp - F)) < 0.02


def test_batched_workload_totals():
    """256 knapsack/cover MIPs with n = 2m and 8 nonzeros per column: 16 m nonzeros
    each, 17.2M in all."""
    sizes = I.power_law_sizes()
    assert len(sizes) == 256
    assert abs(16 * int(sizes.sum()) - 17.2e6) < 0.1e6
    small = I.knapsack_cover(int(sizes.min()), seed=1)
    assert small.nnz == 16 * small.m


def test_mcf_structure_and_feasible_relaxation():
    nodes, deg, K = 12, 4, 4
    inst = I.mcf(nodes=nodes, avg_degree=deg, commodities=K, seed=1)
    arcs = nodes * deg  # each of nodes * deg / 2 edges gives two arcs
    n_links = inst.n - arcs * K - arcs
    assert n_links >= 1 and inst.m == nodes * K + arcs + n_links
    eq = inst.lo == inst.hi
    assert eq[: nodes * K].all() and not eq[nodes * K:].any()
    f = slice(0, arcs * K)
    assert np.all(inst.is_int[f] == 0) and np.all(inst.is_int[arcs * K:] == 1)
    A = inst.csr()
    fh, fl = np.isfinite(inst.hi), np.isfinite(inst.lo)
    Aub = sp.vstack([A[fh], -A[fl]]).tocsr()
    bub = np.concatenate([inst.hi[fh], -inst.lo[fl]])
    r = linprog(inst.c, A_ub=Aub, b_ub=bub, bounds=list(zip(inst.l, inst.u)), method="highs")
    assert r.status == 0


def test_fanout_targets_flip_ten_percent_of_the_binaries():
    inst = I.packing_covering(m=200, n=500, per_col=4, int_frac=0.40, binary=True, seed=4)
    base = np.where(inst.is_int == 1, 1.0, 0.0) * (np.arange(inst.n) % 2)
    T = I.fanout_targets(inst, base, K=8, flip_frac=0.10)
    bins = inst.is_int == 1
    for k in range(8):
        diff = T[:, k] != base
        assert not diff[~bins].any()
        assert diff.sum() == int(round(0.10 * bins.sum()))


def test_open_bounds_lp_recipe():
    """Every column and row kind occurs; the constructed pair is feasible and
    complementary (y_i > 0 only on an active finite lower side, < 0 on an active
    upper side; lambda_j >= 0 at an active lower bound, <= 0 at an upper one, 0
    strictly inside), and c = A^T y* + lambda*."""
    inst = I.open_bounds_lp(400, 800, per_col=6, seed=3)
    x, y = inst.meta["x_star"], inst.meta["y_star"]
    A = inst.csr()
    assert np.all(np.diff(A.tocsc().indptr) == 6)
    assert set(np.unique(inst.meta["col_kind"])) == set(range(len(I.COL_KINDS)))
    assert set(np.unique(inst.meta["row_kind"])) == set(range(len(I.ROW_KINDS)))
    lf, uf = np.isfinite(inst.l), np.isfinite(inst.u)
    assert (lf & ~uf).any() and (~lf & uf).any() and (~lf & ~uf).any() and (inst.l == inst.u).any()
    r = A @ x
    assert np.all(r >= inst.lo - 1e-9) and np.all(r <= inst.hi + 1e-9)
    assert np.all(x >= inst.l) and np.all(x <= inst.u)
    assert np.all(np.isfinite(inst.lo[y > 0])) and np.all(np.isfinite(inst.hi[y < 0]))
    assert np.all(np.abs(r - inst.lo)[y > 0] <= 1e-9 * (1 + np.abs(r[y > 0])))
    assert np.all(np.abs(r - inst.hi)[y < 0] <= 1e-9 * (1 + np.abs(r[y < 0])))
    lam = inst.c - A.T @ y
    inside = (x > inst.l) & (x < inst.u)
    assert np.all(np.abs(lam[inside]) <= 1e-9)
    assert np.all(lam[(x == inst.l) & ~(x == inst.u)] >= -1e-9)
    assert np.all(lam[(x == inst.u) & ~(x == inst.l)] <= 1e-9)
    std = I.standard_form_lp(100, 200, seed=4)
    assert np.all(std.l == 0) and np.all(np.isinf(std.u)) and np.all(std.lo == std.hi)
    assert np.allclose(std.csr() @ std.meta["x_star"], std.lo)
