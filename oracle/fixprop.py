"""ORACLE (test infrastructure only): fix-and-propagate in plain Python FP64.

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may use this module.  It restates Section 2.3 of Scylla (arXiv 2307.03466):
integer variables with fractional values are fixed one at a time to an integer in
their domain, each fix followed by constraint propagation; a constraint that
would empty a domain is ignored from then on; when all integers are fixed, the
remaining variables take their reference value projected onto their domain.  The
output is integral on the integer columns but need not satisfy the rows.

Readings of what Section 2.3 leaves open:

* Fixing order: integer columns sorted by (|xbar_j - round(xbar_j)|, j), most
  integral first; round(v) = floor(v + 1/2); a column already fixed by
  propagation is skipped; the fix value is round(xbar_j) clamped to the domain.
* Propagation: activity-based bound tightening, FIFO row queue.  An initial pass
  queues every row in ascending order.  A row is visited by recomputing its
  minimum and maximum activity from scratch in CSR order (finite parts summed in
  FP64, infinite contributions counted), then deriving candidate bounds for every
  variable of the row from the domains as they were at the start of the visit:
  ``a_j x_j <= hi - (minact - a_j * bound)`` and ``a_j x_j >= lo - (maxact - ...)``.
  Integer candidates are rounded with ``floor(v + 1e-6)`` / ``ceil(v - 1e-6)`` and
  taken when strictly tighter; continuous candidates are taken when finite and
  tighter by more than ``1e-3 * max(1, |old|)``.
* Empty domain: if the row's activity bounds already exclude [lo, hi] by more than
  1e-9, or any candidate would leave ``lb > ub + 1e-9``, the row applies none of
  its changes and is ignored for the rest of the call.  Otherwise all changes are
  applied, and for each changed column (in CSR order) its rows are queued in
  ascending order unless already queued or ignored.
* A propagation call stops after ``visit_cap(m) = 20 m + 1000`` row visits.
* ``propagate_rounds`` is the round-based (Jacobi) form of the same propagation that
  the GPU runs; see its docstring for how rounds merge and when they stop.
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np

INF = math.inf


def visit_cap(m: int) -> int:
    return 20 * m + 1000


class _FixProp:
    def __init__(self, rowptr, cols, vals, lo, hi, l, u, is_int):
        self.m = len(rowptr) - 1
        self.n = len(l)
        self.rowptr = [int(v) for v in rowptr]
        self.cols = [int(v) for v in cols]
        self.vals = [float(v) for v in vals]
        self.lo = [float(v) for v in lo]
        self.hi = [float(v) for v in hi]
        self.dl = [float(v) for v in l]
        self.du = [float(v) for v in u]
        self.is_int = [bool(v) for v in is_int]
        # rows of each column, ascending (the transpose's row lists)
        col_rows = [[] for _ in range(self.n)]
        for i in range(self.m):
            for p in range(self.rowptr[i], self.rowptr[i + 1]):
                col_rows[self.cols[p]].append(i)
        self.col_rows = col_rows
        self.ignored = [False] * self.m
        self.inq = [False] * self.m
        self.queue = deque()
        self.row_visits = 0

    def enqueue(self, i):
        if not self.inq[i] and not self.ignored[i]:
            self.inq[i] = True
            self.queue.append(i)

    def visit(self, i):
        ign, changes = self.proposals(i)
        if ign:
            self.ignored[i] = True
            return
        for j, nl, nu in changes:
            self.dl[j] = nl
            self.du[j] = nu
        for j, _, _ in changes:
            for r in self.col_rows[j]:
                self.enqueue(r)

    def proposals(self, i):
        """(ignore the row, [(j, new_lb, new_ub) for the columns it tightens]) from the
        current domains, without changing them."""
        lo_i, hi_i = self.lo[i], self.hi[i]
        if lo_i == -INF and hi_i == INF:
            return False, []
        dl, du, vals, cols = self.dl, self.du, self.vals, self.cols
        p0, p1 = self.rowptr[i], self.rowptr[i + 1]
        minf = 0.0
        maxf = 0.0
        nmin = 0
        nmax = 0
        for p in range(p0, p1):
            j = cols[p]
            a = vals[p]
            if a > 0:
                bmin, bmax = dl[j], du[j]
            else:
                bmin, bmax = du[j], dl[j]
            if math.isinf(bmin):
                nmin += 1
            else:
                minf += a * bmin
            if math.isinf(bmax):
                nmax += 1
            else:
                maxf += a * bmax
        if nmin == 0 and hi_i != INF and minf > hi_i + 1e-9:
            return True, []
        if nmax == 0 and lo_i != -INF and maxf < lo_i - 1e-9:
            return True, []
        changes = []
        for p in range(p0, p1):
            j = cols[p]
            a = vals[p]
            if a > 0:
                bmin, bmax = dl[j], du[j]
            else:
                bmin, bmax = du[j], dl[j]
            if math.isinf(bmin):
                rmin = minf if nmin == 1 else -INF
            else:
                rmin = (minf - a * bmin) if nmin == 0 else -INF
            if math.isinf(bmax):
                rmax = maxf if nmax == 1 else INF
            else:
                rmax = (maxf - a * bmax) if nmax == 0 else INF
            cand_lb = -INF
            cand_ub = INF
            if hi_i != INF and rmin != -INF:
                t = (hi_i - rmin) / a
                if a > 0:
                    cand_ub = t
                else:
                    cand_lb = t
            if lo_i != -INF and rmax != INF:
                t = (lo_i - rmax) / a
                if a > 0:
                    cand_lb = t
                else:
                    cand_ub = t
            old_lb, old_ub = dl[j], du[j]
            new_lb, new_ub = old_lb, old_ub
            if self.is_int[j]:
                if cand_ub != INF:
                    v = math.floor(cand_ub + 1e-6)
                    if v < old_ub:
                        new_ub = float(v)
                if cand_lb != -INF:
                    v = math.ceil(cand_lb - 1e-6)
                    if v > old_lb:
                        new_lb = float(v)
            else:
                if cand_ub != INF and (old_ub == INF or cand_ub < old_ub - 1e-3 * max(1.0, abs(old_ub))):
                    new_ub = cand_ub
                if cand_lb != -INF and (old_lb == -INF or cand_lb > old_lb + 1e-3 * max(1.0, abs(old_lb))):
                    new_lb = cand_lb
            if new_lb == old_lb and new_ub == old_ub:
                continue
            if new_lb > new_ub + 1e-9:
                return True, []
            changes.append((j, new_lb, new_ub))
        return False, changes

    def propagate(self):
        cap = visit_cap(self.m)
        visits = 0
        while self.queue:
            i = self.queue.popleft()
            self.inq[i] = False
            if self.ignored[i]:
                continue
            if visits >= cap:
                for r in self.queue:
                    self.inq[r] = False
                self.inq[i] = False
                self.queue.clear()
                break
            visits += 1
            self.visit(i)
        self.row_visits += visits


def round_half_up(v: float) -> float:
    return float(math.floor(v + 0.5))


def fixing_order(xbar, is_int):
    """Integer columns sorted by (distance to nearest integer, index)."""
    js = [j for j in range(len(xbar)) if is_int[j]]
    return sorted(js, key=lambda j: (abs(float(xbar[j]) - round_half_up(float(xbar[j]))), j))


def fix_and_propagate(rowptr, cols, vals, lo, hi, l, u, is_int, xbar):
    """Section 2.3.  Returns (xhat, dom_lo, dom_hi, fixed_cols, ignored_rows)."""
    fp = _FixProp(rowptr, cols, vals, lo, hi, l, u, is_int)
    for i in range(fp.m):
        fp.enqueue(i)
    fp.propagate()
    fixed = []
    for j in fixing_order(xbar, is_int):
        if fp.dl[j] == fp.du[j]:
            continue
        v = round_half_up(float(xbar[j]))
        v = min(max(v, fp.dl[j]), fp.du[j])
        fp.dl[j] = v
        fp.du[j] = v
        fixed.append(j)
        for r in fp.col_rows[j]:
            fp.enqueue(r)
        fp.propagate()
    xhat = np.array([min(max(float(xbar[j]), fp.dl[j]), fp.du[j]) for j in range(fp.n)])
    return (xhat, np.array(fp.dl), np.array(fp.du), np.array(fixed, dtype=np.int64),
            np.array(fp.ignored, dtype=bool))


def propagate_rounds(rowptr, cols, vals, lo, hi, l, u, is_int, max_rounds: int = 100000):
    """Propagation in rounds (the order-free form a GPU runs): in each round every
    active row (all rows in the first) computes its proposals from the domains at
    the start of the round, exactly as one FIFO visit does; a row that would empty a
    domain is ignored from then on.  Each column then takes the largest proposed
    lower and the smallest proposed upper bound; if those cross by more than 1e-9
    the column keeps its domain and counts a conflict.  The rows of the columns
    that changed are the next round's active rows.  Stops when no column changes or
    after max_rounds rounds.  On integer data without ignored rows or conflicts this
    is the fixpoint of the FIFO propagation (the greatest fixpoint of a monotone
    tightening; Knaster-Tarski).  Returns (dom_lo, dom_hi, ignored, rounds,
    conflicts)."""
    fp = _FixProp(rowptr, cols, vals, lo, hi, l, u, is_int)
    active = list(range(fp.m))
    rounds = 0
    conflicts = 0
    while active and rounds < max_rounds:
        rounds += 1
        new_l = {}
        new_u = {}
        for i in active:
            if fp.ignored[i]:
                continue
            ign, changes = fp.proposals(i)
            if ign:
                fp.ignored[i] = True
                continue
            for j, nl, nu in changes:
                new_l[j] = max(new_l.get(j, -INF), nl)
                new_u[j] = min(new_u.get(j, INF), nu)
        changed = []
        for j in sorted(set(new_l) | set(new_u)):
            nl = max(fp.dl[j], new_l.get(j, -INF))
            nu = min(fp.du[j], new_u.get(j, INF))
            if nl > nu + 1e-9:
                conflicts += 1
                continue
            if nl != fp.dl[j] or nu != fp.du[j]:
                fp.dl[j] = nl
                fp.du[j] = nu
                changed.append(j)
        nxt = set()
        for j in changed:
            nxt.update(fp.col_rows[j])
        active = sorted(r for r in nxt if not fp.ignored[r])
    return (np.array(fp.dl), np.array(fp.du), np.array(fp.ignored, dtype=bool), rounds, conflicts)


def propagate_only(rowptr, cols, vals, lo, hi, l, u, is_int):
    """The initial propagation pass alone (used by tests).  Returns (dom_lo, dom_hi, ignored)."""
    fp = _FixProp(rowptr, cols, vals, lo, hi, l, u, is_int)
    for i in range(fp.m):
        fp.enqueue(i)
    fp.propagate()
    return np.array(fp.dl), np.array(fp.du), np.array(fp.ignored, dtype=bool)
