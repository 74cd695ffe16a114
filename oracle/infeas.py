"""ORACLE (test infrastructure only): certificates of infeasibility for the LP

    min c^T x   s.t.   lo <= A x <= hi,   l <= x <= u.

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may use this module.  Scylla hands its LP solves to PDLP (Section 2.1), whose solver
also reports infeasible relaxations; these functions state what such a report
rests on, in plain FP64 (``math.fsum``), so that a detector can be checked against
them.  Both are weak duality written out; the detector that proposes the rays is
``PdhgParams.infeasibility_checks`` in oracle/pdhg.py.

* Primal infeasibility (a dual ray y).  For every feasible x,
      sum_i min_{lo_i <= s_i <= hi_i} y_i s_i  <=  y^T A x  =  (A^T y)^T x
                                               <=  sum_j max_{l_j <= x_j <= u_j} (A^T y)_j x_j.
  With D(y) = (left-hand bound) - (right-hand bound), D(y) > 0 proves that no
  feasible x exists.  A term that needs an infinite bound (y_i > 0 with lo_i = -inf,
  (A^T y)_j > 0 with u_j = +inf, and their mirror cases) makes D(y) = -inf: that y
  proves nothing.
* Dual infeasibility (a primal ray d).  If c^T d < 0 and d lies in the recession
  cone of the constraints ((A d)_i >= 0 where lo_i is finite, <= 0 where hi_i is
  finite, d_j >= 0 where l_j is finite, <= 0 where u_j is finite), then from any
  feasible point the objective decreases without bound along d, so the dual has no
  feasible point.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def _side_min(y: np.ndarray, lo: np.ndarray, hi: np.ndarray) -> float:
    """sum_i min over s_i in [lo_i, hi_i] of y_i s_i, -inf if a term is unbounded."""
    terms = []
    for yi, a, b in zip(y, lo, hi):
        if yi > 0:
            if not math.isfinite(a):
                return -math.inf
            terms.append(yi * a)
        elif yi < 0:
            if not math.isfinite(b):
                return -math.inf
            terms.append(yi * b)
    return math.fsum(terms)


def _box_max(r: np.ndarray, l: np.ndarray, u: np.ndarray) -> float:
    """sum_j max over x_j in [l_j, u_j] of r_j x_j, +inf if a term is unbounded."""
    terms = []
    for rj, a, b in zip(r, l, u):
        if rj > 0:
            if not math.isfinite(b):
                return math.inf
            terms.append(rj * b)
        elif rj < 0:
            if not math.isfinite(a):
                return math.inf
            terms.append(rj * a)
    return math.fsum(terms)


def farkas_gap(A, lo, hi, l, u, y) -> float:
    """D(y) of the module docstring: > 0 exactly when y proves the LP infeasible."""
    A = sp.csr_matrix(A)
    y = np.asarray(y, dtype=np.float64)
    r = A.T @ y
    left = _side_min(y, np.asarray(lo, float), np.asarray(hi, float))
    right = _box_max(r, np.asarray(l, float), np.asarray(u, float))
    if left == -math.inf or right == math.inf:
        return -math.inf
    return left - right


def farkas_gap_scale(A, lo, hi, l, u, y):
    """(D(y), S(y)): D as farkas_gap, and S the sum of the absolute values of D's
    terms, the scale against which D's FP64 rounding is small."""
    A = sp.csr_matrix(A)
    y = np.asarray(y, dtype=np.float64)
    lo, hi, l, u = (np.asarray(v, float) for v in (lo, hi, l, u))
    g = farkas_gap(A, lo, hi, l, u, y)
    if g == -math.inf:
        return g, math.inf
    r = A.T @ y
    side = np.where(y > 0, y * np.where(np.isfinite(lo), lo, 0.0), np.where(y < 0, y * np.where(np.isfinite(hi), hi, 0.0), 0.0))
    box = np.where(r > 0, r * np.where(np.isfinite(u), u, 0.0), np.where(r < 0, r * np.where(np.isfinite(l), l, 0.0), 0.0))
    return g, math.fsum(np.abs(side)) + math.fsum(np.abs(box))


def sign_projection(y, lo, hi) -> np.ndarray:
    """y with every entry set to 0 whose sign would need an infinite row side
    (y_i > 0 with lo_i = -inf, y_i < 0 with hi_i = +inf)."""
    y = np.asarray(y, dtype=np.float64)
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    keep = ((y > 0) & np.isfinite(lo)) | ((y < 0) & np.isfinite(hi))
    return np.where(keep, y, 0.0)


def recession_violation(A, lo, hi, l, u, d) -> float:
    """Largest violation of the recession-cone conditions by the direction d (0 when
    d is a recession direction of the feasible set)."""
    A = sp.csr_matrix(A)
    d = np.asarray(d, dtype=np.float64)
    Ad = A @ d
    lo, hi, l, u = (np.asarray(v, float) for v in (lo, hi, l, u))
    v = 0.0
    v = max(v, float(np.max(np.where(np.isfinite(lo), -Ad, 0.0), initial=0.0)))
    v = max(v, float(np.max(np.where(np.isfinite(hi), Ad, 0.0), initial=0.0)))
    v = max(v, float(np.max(np.where(np.isfinite(l), -d, 0.0), initial=0.0)))
    v = max(v, float(np.max(np.where(np.isfinite(u), d, 0.0), initial=0.0)))
    return v


def is_dual_ray(A, c, lo, hi, l, u, d) -> bool:
    """True when d proves the dual infeasible: c^T d < 0 and d a recession direction."""
    cd = math.fsum(np.asarray(c, float) * np.asarray(d, float))
    return cd < 0 and recession_violation(A, lo, hi, l, u, d) == 0.0
