"""Seeded synthetic MIP instances shaped like the workloads of Scylla's evaluation.

The paper evaluates on MIPLIB 2017 and the FP-2.0 instances (Section 3), which are
not available here; these generators stand in for the instances whose LP
relaxations are hard to solve, where Section 3 finds the method most useful.  Every instance is
``min c^T x  s.t.  lo <= A x <= hi,  l <= x <= u,  x_j integer for is_int[j]``,
the two-sided generalisation of the paper's ``A x >= b`` (Algorithm 1, input).

This module only draws random data.  It holds none of the solver's arithmetic and
is the one module that both the CUDA path's tests and the CPU oracle's tests use
for inputs.  All randomness comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

INF = np.inf


@dataclass
class Instance:
    """A MIP in CSR form (row pointers int64, column indices int32, values f64)."""

    name: str
    m: int
    n: int
    rowptr: np.ndarray
    cols: np.ndarray
    vals: np.ndarray
    c: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    l: np.ndarray
    u: np.ndarray
    is_int: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def csr(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.vals, self.cols, self.rowptr), shape=(self.m, self.n))


def _from_coo(name, m, n, rows, cols, vals, c, lo, hi, l, u, is_int, meta=None) -> Instance:
    A = sp.coo_matrix((vals, (rows, cols)), shape=(m, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return Instance(
        name=name, m=m, n=n,
        rowptr=np.ascontiguousarray(A.indptr, dtype=np.int64),
        cols=np.ascontiguousarray(A.indices, dtype=np.int32),
        vals=np.ascontiguousarray(A.data, dtype=np.float64),
        c=np.ascontiguousarray(c, dtype=np.float64),
        lo=np.ascontiguousarray(lo, dtype=np.float64),
        hi=np.ascontiguousarray(hi, dtype=np.float64),
        l=np.ascontiguousarray(l, dtype=np.float64),
        u=np.ascontiguousarray(u, dtype=np.float64),
        is_int=np.ascontiguousarray(is_int, dtype=np.uint8),
        meta=meta or {},
    )


def _distinct_rows_per_column(rng, m: int, n: int, k: int) -> np.ndarray:
    """k distinct uniform row indices for each of n columns, as an (n, k) array."""
    if k > m:
        raise ValueError("k > m")
    out = rng.integers(0, m, size=(n, k))
    # resample duplicates until every column has distinct rows
    for _ in range(64):
        s = np.sort(out, axis=1)
        dup = np.any(s[:, 1:] == s[:, :-1], axis=1)
        if not dup.any():
            return out
        out[dup] = rng.integers(0, m, size=(int(dup.sum()), k))
    raise RuntimeError("could not draw distinct rows")


def set_cover(m: int = 200, n: int = 500, seed: int = 1001, smin: int = 3, smax: int = 8) -> Instance:
    """Random set cover: A x >= 1 with 0/1 coefficients, binary x, costs U{1..100}.

    Column j covers s_j ~ U{smin..smax} distinct rows; a row left uncovered is
    added to a uniformly chosen column.
    """
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    cover = np.zeros(m, dtype=np.int64)
    for j in range(n):
        s = int(rng.integers(smin, smax + 1))
        r = rng.choice(m, size=min(s, m), replace=False)
        rows.append(r)
        cols.append(np.full(len(r), j))
        cover[r] += 1
    for i in np.nonzero(cover == 0)[0]:
        j = int(rng.integers(0, n))
        rows.append(np.array([i]))
        cols.append(np.array([j]))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.ones(len(rows))
    c = rng.integers(1, 101, size=n).astype(np.float64)
    return _from_coo("set_cover", m, n, rows, cols, vals, c,
                     lo=np.ones(m), hi=np.full(m, INF),
                     l=np.zeros(n), u=np.ones(n), is_int=np.ones(n, dtype=np.uint8),
                     meta={"seed": seed})


def _pack_cover_rows(rng, A: sp.csr_matrix, x0: np.ndarray):
    """Row bounds making x0 strictly feasible: half covering, half packing rows."""
    m = A.shape[0]
    r = A @ x0
    s = rng.uniform(0.05, 0.5, size=m)
    covering = rng.random(m) < 0.5
    lo = np.where(covering, r * (1.0 - s), -INF)
    hi = np.where(covering, INF, r * (1.0 + s))
    return lo, hi


def packing_covering(m: int = 50_000, n: int = 100_000, per_col: int = 10,
                     int_frac: float = 0.30, int_ub: float = 10.0, cont_ub: float = 100.0,
                     seed: int = 1002, binary: bool = False, name: str = "pack_cover") -> Instance:
    """Random mixed packing/covering MIP with lognormal(0,1) coefficients.

    ``per_col`` nonzeros per column at distinct uniform rows; a fraction
    ``int_frac`` of the columns are integer in [0, int_ub] (binary when
    ``binary``), the rest continuous in [0, cont_ub].  A random interior point x0
    fixes the row bounds: each row is covering (lo = r(1-s), hi = inf) or packing
    (lo = -inf, hi = r(1+s)) with probability 1/2, s ~ U(0.05, 0.5), r = A x0.
    Objective c_j = +-lognormal(0,1) with a random sign.
    """
    rng = np.random.default_rng(seed)
    rows = _distinct_rows_per_column(rng, m, n, per_col).ravel()
    cols = np.repeat(np.arange(n), per_col)
    vals = rng.lognormal(0.0, 1.0, size=n * per_col)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
    A.sort_indices()
    is_int = (rng.random(n) < int_frac).astype(np.uint8)
    ub_int = 1.0 if binary else int_ub
    u = np.where(is_int == 1, ub_int, cont_ub)
    l = np.zeros(n)
    if binary:
        x0 = np.where(is_int == 1, rng.uniform(0.2, 0.8, size=n), rng.uniform(1.0, cont_ub - 1.0, size=n))
    else:
        x0 = np.where(is_int == 1, rng.integers(1, int(int_ub), size=n).astype(np.float64),
                      rng.uniform(1.0, cont_ub - 1.0, size=n))
    lo, hi = _pack_cover_rows(rng, A, x0)
    sign = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    c = sign * rng.lognormal(0.0, 1.0, size=n)
    return Instance(name=name, m=m, n=n,
                    rowptr=A.indptr.astype(np.int64), cols=A.indices.astype(np.int32),
                    vals=A.data.astype(np.float64), c=c, lo=lo, hi=hi, l=l, u=u, is_int=is_int,
                    meta={"seed": seed, "x0": x0})


def fanout_base(m: int = 200_000, n: int = 500_000, per_col: int = 10, seed: int = 1005) -> Instance:
    """Packing/covering instance with 40% binary columns (the K-objective fan-out base)."""
    return packing_covering(m=m, n=n, per_col=per_col, int_frac=0.40, cont_ub=100.0,
                            seed=seed, binary=True, name="fanout")


def fanout_targets(inst: Instance, base_target: np.ndarray, K: int = 64, flip_frac: float = 0.10,
                   seed: int = 2005) -> np.ndarray:
    """K rounding targets (n x K, column-major per objective) from one base target.

    Each target flips a uniformly random ``flip_frac`` of the binary entries of
    ``base_target`` (1 - value), leaving the rest unchanged.
    """
    rng = np.random.default_rng(seed)
    bins = np.nonzero(inst.is_int == 1)[0]
    nflip = int(round(flip_frac * len(bins)))
    out = np.repeat(base_target[:, None], K, axis=1).astype(np.float64)
    for k in range(K):
        f = rng.choice(bins, size=nflip, replace=False)
        out[f, k] = 1.0 - out[f, k]
    return out


def mcf(nodes: int = 2000, avg_degree: int = 8, commodities: int = 500, link_frac: float = 0.10,
        seed: int = 1003) -> Instance:
    """Multicommodity-flow-shaped MIP relaxation (fixed-charge network design).

    A random Hamiltonian cycle plus uniform random edges up to the average degree,
    each edge giving two arcs.  Variables, in this order: flows f_ak in [0, d_k]
    (arc-major, commodity-minor), arc-open binaries y_a, and binaries z_ak on a
    random ``link_frac`` of the (a, k) pairs.  Rows, in this order: flow
    conservation per (node, commodity) as equalities, capacity rows
    sum_k f_ak - cap_a y_a <= 0, and linking rows f_ak - d_k z_ak <= 0.
    Capacities are max(U{50..500}, load of routing every commodity on one
    shortest path) so the relaxation is feasible.  Costs: flow U{1..10} per arc,
    opening U{100..1000}, z zero.
    """
    from scipy.sparse.csgraph import shortest_path

    rng = np.random.default_rng(seed)
    N = nodes
    target_edges = N * avg_degree // 2
    perm = rng.permutation(N)
    eset = set()
    edges = []
    for i in range(N):
        a, b = int(perm[i]), int(perm[(i + 1) % N])
        key = (min(a, b), max(a, b))
        if key not in eset:
            eset.add(key)
            edges.append(key)
    while len(edges) < target_edges:
        need = target_edges - len(edges)
        cand = rng.integers(0, N, size=(2 * need + 16, 2))
        for a, b in cand:
            if a == b:
                continue
            key = (int(min(a, b)), int(max(a, b)))
            if key in eset:
                continue
            eset.add(key)
            edges.append(key)
            if len(edges) == target_edges:
                break
    e = np.array(edges, dtype=np.int64)
    tail = np.concatenate([e[:, 0], e[:, 1]])
    head = np.concatenate([e[:, 1], e[:, 0]])
    order = np.lexsort((head, tail))
    tail, head = tail[order], head[order]
    n_arcs = len(tail)
    K = commodities
    s_k = rng.integers(0, N, size=K)
    t_k = (s_k + rng.integers(1, N, size=K)) % N
    d_k = rng.integers(1, 51, size=K).astype(np.float64)

    # route each commodity along one (hop-count) shortest path to size capacities
    G = sp.csr_matrix((np.ones(n_arcs), (tail, head)), shape=(N, N))
    arc_id = sp.csr_matrix((np.arange(n_arcs) + 1, (tail, head)), shape=(N, N)).todok()
    srcs = np.unique(s_k)
    _, pred = shortest_path(G, unweighted=True, indices=srcs, return_predecessors=True)
    src_row = {int(s): r for r, s in enumerate(srcs)}
    load = np.zeros(n_arcs)
    for k in range(K):
        p = pred[src_row[int(s_k[k])]]
        v = int(t_k[k])
        while v != int(s_k[k]):
            pv = int(p[v])
            load[int(arc_id[pv, v]) - 1] += d_k[k]
            v = pv
    cap = np.maximum(rng.integers(50, 501, size=n_arcs).astype(np.float64), load)
    arc_cost = rng.integers(1, 11, size=n_arcs).astype(np.float64)
    open_cost = rng.integers(100, 1001, size=n_arcs).astype(np.float64)

    n_f = n_arcs * K
    link = np.nonzero(rng.random(n_f) < link_frac)[0]  # flat (a, k) ids, ascending
    n_z = len(link)
    n = n_f + n_arcs + n_z
    col_f = np.arange(n_f, dtype=np.int64)  # f_ak -> a*K + k
    col_y0 = n_f
    col_z0 = n_f + n_arcs

    # conservation rows: (v, k) -> v*K + k ; +1 on arcs leaving v, -1 on arcs entering v
    a_idx = np.repeat(np.arange(n_arcs, dtype=np.int64), K)
    k_idx = np.tile(np.arange(K, dtype=np.int64), n_arcs)
    r_out = tail[a_idx] * K + k_idx
    r_in = head[a_idx] * K + k_idx
    m_cons = N * K
    rows = [r_out, r_in]
    colsl = [col_f, col_f]
    valsl = [np.ones(n_f), -np.ones(n_f)]
    # capacity rows
    r_cap0 = m_cons
    rows += [r_cap0 + a_idx, r_cap0 + np.arange(n_arcs, dtype=np.int64)]
    colsl += [col_f, col_y0 + np.arange(n_arcs, dtype=np.int64)]
    valsl += [np.ones(n_f), -cap]
    # linking rows
    r_link0 = m_cons + n_arcs
    lr = r_link0 + np.arange(n_z, dtype=np.int64)
    rows += [lr, lr]
    colsl += [link, col_z0 + np.arange(n_z, dtype=np.int64)]
    valsl += [np.ones(n_z), -d_k[link % K]]
    m = m_cons + n_arcs + n_z

    rhs = np.zeros(m_cons)
    rhs[s_k * K + np.arange(K)] += d_k
    rhs[t_k * K + np.arange(K)] -= d_k
    lo = np.concatenate([rhs, np.full(n_arcs + n_z, -INF)])
    hi = np.concatenate([rhs, np.zeros(n_arcs + n_z)])
    c = np.concatenate([np.repeat(arc_cost, K), open_cost, np.zeros(n_z)])
    l = np.zeros(n)
    u = np.concatenate([np.tile(d_k, n_arcs), np.ones(n_arcs), np.ones(n_z)])
    is_int = np.concatenate([np.zeros(n_f, dtype=np.uint8), np.ones(n_arcs + n_z, dtype=np.uint8)])
    return _from_coo("mcf", m, n, np.concatenate(rows), np.concatenate(colsl), np.concatenate(valsl),
                     c, lo, hi, l, u, is_int,
                     meta={"seed": seed, "nodes": N, "arcs": n_arcs, "commodities": K})


def knapsack_cover(m: int, seed: int, per_col: int = 8) -> Instance:
    """Covering/knapsack-mix MIP: n = 2m binary columns, integer coefficients U{1..20}.

    x0 ~ Bernoulli(1/2); each row is a knapsack (hi = (A x0)_i + floor(0.1 rowsum))
    or a cover (lo = max(1, (A x0)_i - floor(0.1 rowsum))) with probability 1/2.
    Objective c_j ~ U{-10..10} without 0.
    """
    rng = np.random.default_rng(seed)
    n = 2 * m
    k = min(per_col, m)
    rows = _distinct_rows_per_column(rng, m, n, k).ravel()
    cols = np.repeat(np.arange(n), k)
    vals = rng.integers(1, 21, size=n * k).astype(np.float64)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
    A.sort_indices()
    x0 = (rng.random(n) < 0.5).astype(np.float64)
    r = A @ x0
    rowsum = np.asarray(A.sum(axis=1)).ravel()
    slack = np.floor(0.1 * rowsum)
    knap = rng.random(m) < 0.5
    lo = np.where(knap, -INF, np.maximum(1.0, r - slack))
    hi = np.where(knap, r + slack, INF)
    c = rng.integers(1, 11, size=n).astype(np.float64) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return Instance(name="knapsack_cover", m=m, n=n,
                    rowptr=A.indptr.astype(np.int64), cols=A.indices.astype(np.int32),
                    vals=A.data.astype(np.float64), c=c, lo=lo, hi=hi,
                    l=np.zeros(n), u=np.ones(n), is_int=np.ones(n, dtype=np.uint8),
                    meta={"seed": seed})


def power_law_sizes(count: int = 256, m_min: int = 1000, m_max: int = 50_000, seed: int = 1004) -> np.ndarray:
    """Row counts from p(m) proportional to m^-2 on [m_min, m_max] by inverse CDF."""
    rng = np.random.default_rng(seed)
    uu = rng.random(count)
    inv = 1.0 / m_min - uu * (1.0 / m_min - 1.0 / m_max)
    return np.maximum(m_min, np.minimum(m_max, np.floor(1.0 / inv))).astype(np.int64)


def batch(count: int = 256, m_min: int = 1000, m_max: int = 50_000, seed: int = 1004) -> list:
    """The batched workload: ``count`` knapsack/cover MIPs with power-law sizes."""
    sizes = power_law_sizes(count, m_min, m_max, seed)
    return [knapsack_cover(int(mb), seed=seed * 1000 + b) for b, mb in enumerate(sizes)]


def tiny_lp(seed: int, m: int = 4, n: int = 5, density: float = 0.6, int_data: bool = False,
            box: float = 4.0) -> Instance:
    """A small random LP with finite boxes, for brute-force checks."""
    rng = np.random.default_rng(seed)
    dense = np.where(rng.random((m, n)) < density,
                     rng.integers(-3, 4, size=(m, n)) if int_data else rng.normal(size=(m, n)), 0.0)
    for i in range(m):
        if not dense[i].any():
            dense[i, rng.integers(0, n)] = 1.0
    x0 = rng.uniform(0.5, box - 0.5, size=n)
    r = dense @ x0
    kind = rng.integers(0, 4, size=m)  # 0 >=, 1 <=, 2 ranged, 3 equality
    s = rng.uniform(0.2, 1.0, size=m)
    lo = np.where(kind == 1, -INF, np.where(kind == 3, r, r - s))
    hi = np.where(kind == 0, INF, np.where(kind == 3, r, r + s))
    A = sp.csr_matrix(dense)
    A.eliminate_zeros()
    A.sort_indices()
    c = rng.normal(size=n)
    return Instance(name="tiny", m=m, n=n, rowptr=A.indptr.astype(np.int64),
                    cols=A.indices.astype(np.int32), vals=A.data.astype(np.float64),
                    c=c, lo=lo, hi=hi, l=np.zeros(n), u=np.full(n, box),
                    is_int=np.zeros(n, dtype=np.uint8), meta={"seed": seed, "dense": dense})


# column kinds of open_bounds_lp: boxed [l, u], lower-bounded only [l, inf),
# upper-bounded only (-inf, u], free, fixed (l = u)
COL_KINDS = ("boxed", "lower", "upper", "free", "fixed")
# row kinds: covering [lo, inf), packing (-inf, hi], ranged [lo, hi], equality, free
ROW_KINDS = ("covering", "packing", "ranged", "equality", "free")


def open_bounds_lp(m: int, n: int, per_col: int = 6, seed: int = 0, col_mix=None, row_mix=None,
                   name: str = "open_bounds") -> Instance:
    """LP with one-sided, free and fixed columns and every row kind, built around a
    known optimal primal-dual pair so that its optimum is finite and known.

    A has ``per_col`` nonzeros per column at distinct uniform rows with values
    +-lognormal(0, 1).  Column kinds are drawn with the weights ``col_mix`` (a dict
    over COL_KINDS) and row kinds with ``row_mix`` (over ROW_KINDS).  The pair is
    drawn first: x* at a bound or strictly inside it, y* and the reduced costs
    lambda* with the signs that make both complementary (y*_i > 0 only where lo_i is
    finite and active, < 0 only where hi_i is, 0 on an inactive row; lambda*_j >= 0 at
    an active lower bound, <= 0 at an active upper bound, 0 inside, either sign on a
    fixed column).  Then lo, hi are set at or away from A x*, and c = A^T y* + lambda*.
    (x*, y*) satisfies the optimality conditions of the LP, so f* = c^T x* is its
    optimal value (meta "x_star", "y_star", "f_star").  Data only: no solver step.
    """
    rng = np.random.default_rng(seed)
    cm = dict(boxed=0.3, lower=0.3, upper=0.1, free=0.2, fixed=0.1) if col_mix is None else dict(col_mix)
    rm = dict(covering=0.3, packing=0.3, ranged=0.2, equality=0.15, free=0.05) if row_mix is None else dict(row_mix)
    cw = np.array([cm.get(k, 0.0) for k in COL_KINDS], float)
    rw = np.array([rm.get(k, 0.0) for k in ROW_KINDS], float)
    ck = rng.choice(len(COL_KINDS), size=n, p=cw / cw.sum())
    rk = rng.choice(len(ROW_KINDS), size=m, p=rw / rw.sum())
    k = min(per_col, m)
    rows = _distinct_rows_per_column(rng, m, n, k).ravel()
    cols = np.repeat(np.arange(n), k)
    vals = rng.lognormal(0.0, 1.0, size=n * k) * np.where(rng.random(n * k) < 0.5, -1.0, 1.0)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(m, n))
    A.sort_indices()
    # columns: bounds, x*, lambda*
    l = np.full(n, -INF)
    u = np.full(n, INF)
    x = np.zeros(n)
    lam = np.zeros(n)
    pos = rng.integers(0, 3, size=n)  # 0 at lower, 1 at upper, 2 inside
    mag = rng.uniform(0.1, 2.0, size=n)
    gap = rng.uniform(0.5, 5.0, size=n)
    lb = rng.uniform(-3.0, 3.0, size=n)
    for j in range(n):
        kind = COL_KINDS[ck[j]]
        if kind == "boxed":
            l[j] = lb[j]
            u[j] = lb[j] + 1.0 + gap[j]
            x[j] = l[j] if pos[j] == 0 else (u[j] if pos[j] == 1 else l[j] + 0.5 * (u[j] - l[j]))
            lam[j] = mag[j] if pos[j] == 0 else (-mag[j] if pos[j] == 1 else 0.0)
        elif kind == "lower":
            l[j] = lb[j]
            at = pos[j] != 2
            x[j] = l[j] if at else l[j] + gap[j]
            lam[j] = mag[j] if at else 0.0
        elif kind == "upper":
            u[j] = lb[j]
            at = pos[j] != 2
            x[j] = u[j] if at else u[j] - gap[j]
            lam[j] = -mag[j] if at else 0.0
        elif kind == "free":
            x[j] = rng.uniform(-5.0, 5.0)
        else:  # fixed
            l[j] = u[j] = x[j] = lb[j]
            lam[j] = rng.normal()
    # rows: bounds around r = A x*, y*
    r = A @ x
    lo = np.full(m, -INF)
    hi = np.full(m, INF)
    y = np.zeros(m)
    act = rng.random(m) < 0.5
    ym = rng.uniform(0.1, 2.0, size=m)
    s = rng.uniform(0.1, 1.0, size=m) * (1.0 + np.abs(r))
    side = rng.random(m) < 0.5
    for i in range(m):
        kind = ROW_KINDS[rk[i]]
        if kind == "covering":
            lo[i] = r[i] if act[i] else r[i] - s[i]
            y[i] = ym[i] if act[i] else 0.0
        elif kind == "packing":
            hi[i] = r[i] if act[i] else r[i] + s[i]
            y[i] = -ym[i] if act[i] else 0.0
        elif kind == "ranged":
            if act[i] and side[i]:
                lo[i], hi[i], y[i] = r[i], r[i] + s[i], ym[i]
            elif act[i]:
                lo[i], hi[i], y[i] = r[i] - s[i], r[i], -ym[i]
            else:
                lo[i], hi[i] = r[i] - s[i], r[i] + 0.5 * s[i]
        elif kind == "equality":
            lo[i] = hi[i] = r[i]
            y[i] = rng.normal()
    c = A.T @ y + lam
    return Instance(name=name, m=m, n=n, rowptr=A.indptr.astype(np.int64), cols=A.indices.astype(np.int32),
                    vals=A.data.astype(np.float64), c=np.asarray(c, np.float64), lo=lo, hi=hi, l=l, u=u,
                    is_int=np.zeros(n, dtype=np.uint8),
                    meta={"seed": seed, "x_star": x, "y_star": y, "f_star": float(np.dot(c, x)),
                          "col_kind": ck, "row_kind": rk})


def standard_form_lp(m: int, n: int, per_col: int = 6, seed: int = 0) -> Instance:
    """open_bounds_lp in standard form: every column x_j >= 0 (u = +inf, l = 0 after
    the shift below) and every row an equality."""
    inst = open_bounds_lp(m, n, per_col, seed, col_mix={"lower": 1.0}, row_mix={"equality": 1.0},
                          name="standard_form")
    # shift x -> x - l so that every lower bound is 0: the rows move by A l
    A = inst.csr()
    shift = A @ inst.l
    inst.lo = inst.lo - shift
    inst.hi = inst.hi - shift
    inst.meta["x_star"] = inst.meta["x_star"] - inst.l
    inst.meta["f_star"] = float(np.dot(inst.c, inst.meta["x_star"]))
    inst.l = np.zeros(n)
    return inst


CONFIGS = {
    "setcover_200x500": lambda: set_cover(),
    "packcover_50kx100k": lambda: packing_covering(),
    "mcf_2000n_500k": lambda: mcf(),
    "fanout_200kx500k": lambda: fanout_base(),
}
