"""ORACLE (test infrastructure only): the Scylla outer loop in plain Python FP64.

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may use this module.  It restates Algorithm 1 of Scylla (arXiv 2307.03466): PDHG
with the tolerance schedule of Section 2.2, the MIP-feasibility tests, fix-and-
propagate (Section 2.3), cycle handling by random perturbation (Section 2.3) and
the objective update of Section 2.4.

Readings of what the paper leaves open:

* Tolerance schedule (Section 2.2): eps^(1) = 0.01, eps^(K+1) = max(0.98 eps^(K), 1e-8).
* Objective update (Algorithm 1, Section 2.4): ``c_hat = alpha^K s c + (1 - alpha^K)
  Delta(x, xhat)`` with alpha = 0.9, s = sqrt(|I|) / ||c||_2 (0 when c = 0) and the
  l1 distance Delta over the integer columns.  A column with u - l = 1 contributes
  ``x_j - l_j`` (xhat_j = l_j) or ``u_j - x_j`` (xhat_j = u_j).  Any other integer
  column j gets an auxiliary column d_j in [0, u_j - l_j] with two rows
  ``d_j - x_j >= -xhat_j`` and ``d_j + x_j >= xhat_j`` (Section 4 notes that the l1
  distance on general integers needs auxiliary variables); d_j has cost
  (1 - alpha^K).  Auxiliary columns follow the original columns, auxiliary rows
  follow the original rows, both in ascending j; before the first update the
  auxiliary rows are free (lo = -inf) and cost 0.  Constants of Delta go into the
  objective offset.
* l2 distance (``distance = 2``; the paper's conclusion proposes it for avoiding the
  auxiliary variables): ``alpha^K s c^T x + (1 - alpha^K) 1/2 sum_I (x_j - xhat_j)^2``
  on every integer column, solved as a diagonal-Hessian PDHG (``OracleLP``'s
  quadratic mode); no auxiliary columns.
* MIP-feasible xbar (Algorithm 1): round the integer entries to nearest; accept
  when every one was within 1e-6 and the rounded point passes ``check_feasible``.
* Cycling (Section 2.3, following Fischetti-Glover-Lodi 2005): a short cycle
  (xhat^(K) equal to xhat^(K-1) on I) flips the TT integer columns with largest
  |xbar_j - xhat_j| > 0 (ties: lower j), TT ~ U{10..30}; a long cycle (equal to an
  older one), or a short one with nothing to flip, flips column j when
  ``|xbar_j - xhat_j| + max(rho_j, 0) > 0.5``, rho_j ~ U[-0.3, 0.7].  A flip moves
  one unit toward xbar_j, or away from it when xhat_j already is round(xbar_j),
  inside [l_j, u_j] (the other direction when the first one is blocked).  Random
  numbers: SplitMix64 seeded with ``seed XOR K``, uniforms ``(r >> 11) * 2^-53``.
* Continuous repair (an extension; the paper keeps the continuous part of the
  fix-and-propagate point at the LP values, Section 2.3): the fixing is first
  propagated in rounds (``fixprop.propagate_rounds``, at most 1000); a row it
  ignores or a conflict proves the fixed LP infeasible and ends the repair (no
  solve; x = xhat clamped to the bounds).  Otherwise the LP of the original
  MIP with every integer column fixed at xhat (l_j = u_j = xhat_j), original
  objective and rows, is solved by the oracle PDHG to the given rel-KKT in up to
  ``rounds`` solves (the first from the cold start, the next ones warm) within one
  attempt budget.  After each solve the integer entries are set to xhat's and the
  point is given the feasibility check; when it fails, every row whose activity
  (FP64, CSR order) exceeds an original bound gets its working bound moved inward
  by the excess plus 1e-6 max(1, |bound|) (crossing working bounds meet at their
  midpoint), since a PDHG point can miss single rows by more than the check's
  tolerance long after its relative KKT error is small.  In the outer loop the
  repair runs, when asked for, after a fix-and-propagate point fails the check and
  before the cycle test.
* Feasibility check: integrality exact; a row whose coefficients, bounds and
  column values are all integers of magnitude below 2^47 is checked in exact
  integer arithmetic (the library sums such rows in 128-bit integers: products stay
  below 2^94 and a row of fewer than 2^31 of them below 2^125, so no sum can
  overflow; this oracle uses the same limit so that both take the same branch); otherwise activities are summed in CSR order with Neumaier
  compensation and compared with tolerance 1e-6 * max(1, |bound|).  Continuous
  column bounds use the same tolerance, integer column bounds are exact.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import fixprop
from .pdhg import OracleLP, PdhgParams

INF = math.inf
MASK64 = (1 << 64) - 1
FOUND, NOT_FOUND = 0, 1


def eps_schedule(K: int, eps1: float = 0.01, beta: float = 0.98, floor: float = 1e-8) -> float:
    """eps^(K) of Section 2.2 by its recursion."""
    e = eps1
    for _ in range(K - 1):
        e = max(beta * e, floor)
    return e


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next() >> 11) * (2.0 ** -53)


def general_integer_columns(is_int, l, u):
    """Integer columns that need an auxiliary distance column (u - l != 1)."""
    return [j for j in range(len(l)) if is_int[j] and not (u[j] - l[j] == 1.0)]


@dataclass
class Augmented:
    A: sp.csr_matrix
    c: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    l: np.ndarray
    u: np.ndarray
    n_orig: int
    m_orig: int
    gen_int: list


def augment(A: sp.csr_matrix, c, lo, hi, l, u, is_int) -> Augmented:
    """Append the auxiliary columns and rows for the l1 distance on general integers."""
    m, n = A.shape
    gi = general_integer_columns(is_int, l, u)
    na = len(gi)
    if na == 0:
        return Augmented(sp.csr_matrix(A), np.array(c, float), np.array(lo, float), np.array(hi, float),
                         np.array(l, float), np.array(u, float), n, m, gi)
    rows, cols, vals = [], [], []
    for t, j in enumerate(gi):
        # row m+2t: d_t - x_j ; row m+2t+1: d_t + x_j
        rows += [2 * t, 2 * t, 2 * t + 1, 2 * t + 1]
        cols += [j, n + t, j, n + t]
        vals += [-1.0, 1.0, 1.0, 1.0]
    B = sp.csr_matrix((vals, (rows, cols)), shape=(2 * na, n + na))
    A2 = sp.vstack([sp.hstack([A, sp.csr_matrix((m, na))]), B]).tocsr()
    A2.sort_indices()
    c2 = np.concatenate([np.asarray(c, float), np.zeros(na)])
    lo2 = np.concatenate([np.asarray(lo, float), np.full(2 * na, -INF)])
    hi2 = np.concatenate([np.asarray(hi, float), np.full(2 * na, INF)])
    l2 = np.concatenate([np.asarray(l, float), np.zeros(na)])
    u2 = np.concatenate([np.asarray(u, float), np.array([u[j] - l[j] for j in gi], float)])
    return Augmented(A2, c2, lo2, hi2, l2, u2, n, m, gi)


def objective_update(c, is_int, l, u, xhat, K, gen_int, alpha=0.9):
    """c_hat, auxiliary-row lower bounds and objective offset for round K >= 1."""
    n = len(c)
    aK = alpha ** K
    om = 1.0 - aK
    nI = int(sum(1 for j in range(n) if is_int[j]))
    cn = math.sqrt(sum(float(v) * float(v) for v in c))
    s = math.sqrt(nI) / cn if cn > 0 else 0.0
    t = aK * s
    gen = set(gen_int)
    chat = np.zeros(n + len(gen_int))
    offset = 0.0
    for j in range(n):
        g = 0.0
        if is_int[j] and j not in gen:
            if xhat[j] == l[j]:
                g = 1.0
                offset -= om * l[j]
            elif xhat[j] == u[j]:
                g = -1.0
                offset += om * u[j]
        chat[j] = t * c[j] + om * g
    aux_lo = np.zeros(2 * len(gen_int))
    for q, j in enumerate(gen_int):
        chat[n + q] = om
        aux_lo[2 * q] = -xhat[j]
        aux_lo[2 * q + 1] = xhat[j]
    return chat, aux_lo, offset


def objective_update_l2(c, is_int, xhat, K, alpha=0.9):
    """The l2-distance objective of round K >= 1 (the conclusion's alternative to the
    l1 distance, which needs no auxiliary columns):
        alpha^K s c^T x + (1 - alpha^K) 1/2 sum_{j in I} (x_j - xhat_j)^2
      = c_hat^T x + 1/2 x^T diag(q) x + offset,
    c_hat_j = alpha^K s c_j - (1 - alpha^K) xhat_j and q_j = 1 - alpha^K on I,
    c_hat_j = alpha^K s c_j and q_j = 0 elsewhere, offset = (1 - alpha^K)/2 sum_I xhat_j^2,
    with s = sqrt(|I|) / ||c||_2 (0 when c = 0) as in the l1 update."""
    n = len(c)
    aK = alpha ** K
    om = 1.0 - aK
    nI = int(sum(1 for j in range(n) if is_int[j]))
    cn = math.sqrt(sum(float(v) * float(v) for v in c))
    s = math.sqrt(nI) / cn if cn > 0 else 0.0
    t = aK * s
    chat = np.zeros(n)
    q = np.zeros(n)
    offset = 0.0
    for j in range(n):
        if is_int[j]:
            chat[j] = t * c[j] - om * xhat[j]
            q[j] = om
            offset += 0.5 * om * xhat[j] * xhat[j]
        else:
            chat[j] = t * c[j]
    return chat, q, offset


def _flip(v, xb, lj, uj):
    r = math.floor(xb + 0.5)
    s = 1.0 if xb >= v else -1.0
    if v == r:
        s = -s
    for d in (s, -s):
        w = v + d
        if lj <= w <= uj:
            return w
    return v


def perturb(xhat, xbar, history, K, seed, int_cols, l, u):
    """Cycle test and perturbation (Algorithm 1, Section 2.3).  Returns (xhat, kind)."""
    key = tuple(float(xhat[j]) for j in int_cols)
    if not history:
        return xhat, "none"
    short = key == history[-1]
    long_ = (not short) and key in set(history[:-1])
    if not short and not long_:
        return xhat, "none"
    x = np.array(xhat, dtype=np.float64)
    rng = SplitMix64(seed ^ K)
    if short:
        TT = 10 + int(math.floor(rng.uniform() * 21))
        sig = [(abs(float(xbar[j]) - float(x[j])), j) for j in int_cols]
        cand = sorted([(sv, j) for sv, j in sig if sv > 0], key=lambda t: (-t[0], t[1]))
        if cand:
            for _, j in cand[:TT]:
                x[j] = _flip(float(x[j]), float(xbar[j]), float(l[j]), float(u[j]))
            return x, "short"
    for j in int_cols:
        rho = -0.3 + rng.uniform()
        if abs(float(xbar[j]) - float(x[j])) + max(rho, 0.0) > 0.5:
            x[j] = _flip(float(x[j]), float(xbar[j]), float(l[j]), float(u[j]))
    return x, "long"


def _neumaier(terms):
    s = 0.0
    comp = 0.0
    for t in terms:
        tt = s + t
        if abs(s) >= abs(t):
            comp += (s - tt) + t
        else:
            comp += (t - tt) + s
        s = tt
    return s + comp


def _is_int_val(v):
    return math.isfinite(v) and v == math.floor(v) and abs(v) < 2.0 ** 47


def check_feasible(rowptr, cols, vals, lo, hi, l, u, is_int, x, tol=1e-6) -> bool:
    """Exact MIP-feasibility test of x (see module docstring)."""
    n = len(l)
    for j in range(n):
        v = float(x[j])
        if not math.isfinite(v):
            return False
        if is_int[j]:
            if v != math.floor(v) or v < l[j] or v > u[j]:
                return False
        else:
            if v < l[j] - tol * max(1.0, abs(l[j])) or v > u[j] + tol * max(1.0, abs(u[j])):
                return False
    m = len(rowptr) - 1
    for i in range(m):
        p0, p1 = int(rowptr[i]), int(rowptr[i + 1])
        lo_i, hi_i = float(lo[i]), float(hi[i])
        exact = ((lo_i == -INF or _is_int_val(lo_i)) and (hi_i == INF or _is_int_val(hi_i))
                 and all(_is_int_val(float(vals[p])) and _is_int_val(float(x[cols[p]])) for p in range(p0, p1)))
        if exact:
            act = sum(int(vals[p]) * int(x[cols[p]]) for p in range(p0, p1))
            if lo_i != -INF and act < int(lo_i):
                return False
            if hi_i != INF and act > int(hi_i):
                return False
        else:
            act = _neumaier([float(vals[p]) * float(x[cols[p]]) for p in range(p0, p1)])
            if lo_i != -INF and act < lo_i - tol * max(1.0, abs(lo_i)):
                return False
            if hi_i != INF and act > hi_i + tol * max(1.0, abs(hi_i)):
                return False
    return True


def repair(inst, xhat, tol: float, iter_limit: int, params: PdhgParams | None = None, rounds: int = 8):
    """Continuous repair of xhat's integer assignment (see the module notes).
    Returns (status FOUND / NOT_FOUND, x, dict of iterations, rounds, shifted_rows,
    rel_kkt and status of the last solve)."""
    A = sp.csr_matrix((inst.vals, inst.cols, inst.rowptr), shape=(inst.m, inst.n))
    is_int = np.asarray(inst.is_int) == 1
    xh = np.asarray(xhat, dtype=np.float64)
    l = np.asarray(inst.l, dtype=np.float64).copy()
    u = np.asarray(inst.u, dtype=np.float64).copy()
    l[is_int] = xh[is_int]
    u[is_int] = xh[is_int]
    lo = np.asarray(inst.lo, dtype=np.float64)
    hi = np.asarray(inst.hi, dtype=np.float64)
    info = {"iterations": 0, "rounds": 0, "shifted_rows": 0, "rel_kkt": math.inf, "status": None}
    _, _, ign, _, conf = fixprop.propagate_rounds(inst.rowptr, inst.cols, inst.vals, lo, hi, l, u, inst.is_int,
                                                  max_rounds=1000)
    if ign.any() or conf > 0:
        return NOT_FOUND, np.minimum(np.maximum(xh, l), u), info
    lo_w, hi_w = lo.copy(), hi.copy()
    lp = OracleLP(A, inst.c, lo_w, hi_w, l, u, params=params or PdhgParams())
    st = NOT_FOUND
    x = None
    for t in range(rounds):
        res = lp.solve(tol, iter_limit - info["iterations"])
        info["iterations"] += res.iterations
        info["rounds"] = t + 1
        info["rel_kkt"] = res.rel_kkt
        info["status"] = res.status
        x = lp.primal().copy()
        x[is_int] = xh[is_int]
        if check_feasible(inst.rowptr, inst.cols, inst.vals, lo, hi, inst.l, inst.u, inst.is_int, x):
            st = FOUND
            break
        if t + 1 == rounds or info["iterations"] >= iter_limit:
            break
        act = A @ x
        up = act > hi
        dn = (act < lo) & ~up
        hi_w[up] -= (act[up] - hi[up]) + 1e-6 * np.maximum(1.0, np.abs(hi[up]))
        lo_w[dn] += (lo[dn] - act[dn]) + 1e-6 * np.maximum(1.0, np.abs(lo[dn]))
        cross = (up | dn) & (lo_w > hi_w)
        mid = 0.5 * (lo_w[cross] + hi_w[cross])
        lo_w[cross] = mid
        hi_w[cross] = mid
        info["shifted_rows"] += int(np.count_nonzero(up | dn))
        lp.set_row_bounds(lo_w, hi_w)
    return st, x, info


@dataclass
class PumpParams:
    alpha: float = 0.9
    eps1: float = 0.01
    beta: float = 0.98
    eps_floor: float = 1e-8
    max_rounds: int = 100
    iter_limit: int = 20000
    total_iter_cap: int = 10 ** 9
    stall_checks: int = 5
    seed: int = 0
    repair_iters: int = 0  # attempt limit of each continuous repair; 0 = none
    repair_tol: float = 1e-7
    repair_rounds: int = 8
    distance: int = 1  # 1: l1 distance (Algorithm 1, auxiliary columns on general integers); 2: l2
    pdhg: PdhgParams = field(default_factory=PdhgParams)


@dataclass
class PumpResult:
    status: int
    x: np.ndarray | None
    rounds: int
    total_iterations: int
    found_by: str
    log: list


def pump(inst, params: PumpParams | None = None) -> PumpResult:
    """Algorithm 1 on an ``instances.Instance``-like object (fields rowptr, cols, vals,
    c, lo, hi, l, u, is_int, m, n)."""
    pp = params or PumpParams()
    A = sp.csr_matrix((inst.vals, inst.cols, inst.rowptr), shape=(inst.m, inst.n))
    l2 = pp.distance == 2
    if l2:  # no auxiliary columns: the LP as given
        aug = Augmented(A, np.asarray(inst.c, float), np.asarray(inst.lo, float), np.asarray(inst.hi, float),
                        np.asarray(inst.l, float), np.asarray(inst.u, float), inst.n, inst.m, [])
    else:
        aug = augment(A, inst.c, inst.lo, inst.hi, inst.l, inst.u, inst.is_int)
    int_cols = [j for j in range(inst.n) if inst.is_int[j]]
    pd = PdhgParams(**{**pp.pdhg.__dict__, "stall_checks": pp.stall_checks})
    lp = OracleLP(aug.A, aug.c, aug.lo, aug.hi, aug.l, aug.u, int_cols=int_cols, params=pd)
    hist = []
    K = 1
    eps = pp.eps1
    total = 0
    log = []
    n = inst.n
    while K <= pp.max_rounds and total < pp.total_iter_cap:
        res = lp.solve(eps, min(pp.iter_limit, pp.total_iter_cap - total))
        total += res.iterations
        xbar = lp.primal()[:n]
        xr = xbar.copy()
        near = True
        for j in int_cols:
            r = math.floor(xbar[j] + 0.5)
            if abs(xbar[j] - r) > 1e-6:
                near = False
            xr[j] = r
        if near and check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u,
                                   inst.is_int, xr):
            return PumpResult(FOUND, xr, K, total, "lp", log)
        xhat, _, _, _, _ = fixprop.fix_and_propagate(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi,
                                                     inst.l, inst.u, inst.is_int, xbar)
        if check_feasible(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u,
                          inst.is_int, xhat):
            return PumpResult(FOUND, xhat, K, total, "fixprop", log)
        if pp.repair_iters > 0:
            st, xrep, rinfo = repair(inst, xhat, pp.repair_tol, min(pp.repair_iters, pp.total_iter_cap - total),
                                     pp.pdhg, pp.repair_rounds)
            total += rinfo["iterations"]
            if st == FOUND:
                return PumpResult(FOUND, xrep, K, total, "repair", log)
        xhat, kind = perturb(xhat, xbar, hist, K, pp.seed, int_cols, inst.l, inst.u)
        hist.append(tuple(float(xhat[j]) for j in int_cols))
        if l2:
            chat, q, offset = objective_update_l2(inst.c, inst.is_int, xhat, K, pp.alpha)
            lp.set_objective_vector(chat, offset)
            lp.set_quadratic(q)
            log.append((K, res.status, res.iterations, res.rel_kkt, kind))
            eps = max(pp.beta * eps, pp.eps_floor)
            K += 1
            continue
        chat, aux_lo, offset = objective_update(inst.c, inst.is_int, inst.l, inst.u, xhat, K,
                                                aug.gen_int, pp.alpha)
        lp.set_objective_vector(chat, offset)
        if len(aug.gen_int):
            lo2 = lp.lo.copy()
            lo2[aug.m_orig:] = aux_lo
            lp.set_row_bounds(lo2, lp.hi)
        log.append((K, res.status, res.iterations, res.rel_kkt, kind))
        eps = max(pp.beta * eps, pp.eps_floor)
        K += 1
    return PumpResult(NOT_FOUND, None, K - 1, total, "", log)
