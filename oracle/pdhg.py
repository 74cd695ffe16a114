"""ORACLE (test infrastructure only): plain FP64 PDHG for the LP relaxation.

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may use this module.  It follows Algorithm 1 of Scylla (arXiv 2307.03466): the
primal step ``d_x = A^T y - c_hat, x' = proj_[l,u](x + tau_x d_x)`` and the dual
step ``d_y = b - A(2x' - x), y' = proj(y + tau_y d_y)``, with the step-size,
restart, averaging and preconditioning rules of PDLP that Section 2.1 delegates to
(the paper gives none of them; the readings are listed below), and the stopping
rule of Section 2.2 (relative KKT error against a tolerance).

Readings of points the paper leaves open (each is a parameter):

* Two-sided rows ``lo <= Ax <= hi`` generalise ``Ax >= b``.  The dual step is the
  proximal step of the row-bound support function; for a component
  ``t_lo = y + tau_y (lo - Ax~)``, ``t_hi = y + tau_y (hi - Ax~)``:
  ``y' = t_lo`` if lo is finite and ``t_lo > 0``, else ``t_hi`` if hi is finite and
  ``t_hi < 0``, else 0.  With ``lo = b, hi = +inf`` this is exactly the paper's
  ``max(0, y + tau_y (b - A(2x'-x)))`` (projection onto the non-negative orthant of
  R^m; the paper's R^n is read as R^m).
* Initial point ``x = proj_[l,u](0)``, ``y = 0`` (Algorithm 1 initialises x = 0).
* ``tau_x = eta / omega``, ``tau_y = eta * omega``; ``eta`` is chosen by the
  adaptive rule (step-size update line of Algorithm 1), ``omega`` is the primal
  weight.  Fixed-step mode uses ``eta = f / ||A~||_F`` and never rejects.
* The iteration counter ``k`` counts step attempts of one solve.  The step-size
  rule ``eta' = min((1 - (k+1)^-0.3) eta_max, (1 + (k+1)^-0.6) eta)`` uses the
  1-based number k of the attempt being made (k = 0 would zero the step).  Every
  ``n_check`` attempts, and at the iteration limit, the current and the averaged
  iterate are evaluated; termination, restart and stall decisions are taken there.
* Preconditioning: Ruiz equilibration then Pock-Chambolle (alpha = 1); the
  iteration runs on the scaled LP, residual norms for termination are measured on
  the original one.
* Diagonal quadratic objectives (the conclusion's MIQP remark and its l2 distance:
  PDHG with a diagonal Hessian, as in PDLP): ``min c^T x + 1/2 x^T diag(q) x``,
  q >= 0.  The primal step becomes the closed-form prox of the quadratic plus the
  box, ``x' = proj_[l,u]((x + tau_x (A^T y - c)) / (1 + tau_x q))`` on the scaled
  problem (q~ = q C^2); the dual step is unchanged.  In the KKT error the reduced
  cost is ``c + q x - A^T y``, the primal objective gains ``+1/2 x^T Q x`` and the
  dual objective ``-1/2 x^T Q x``.  q = 0 is the LP exactly.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from oracle import infeas

INF = math.inf

CONVERGED, ITER_LIMIT, STALLED, INFEASIBLE = 0, 1, 2, 3

MASK64 = (1 << 64) - 1


@dataclass
class PdhgParams:
    n_check: int = 64
    ruiz_iters: int = 10
    pock_chambolle: bool = True
    adaptive_step: bool = True
    restarts: bool = True
    primal_weight_update: bool = True
    fixed_step_factor: float = 0.9
    beta_sufficient: float = 0.2
    beta_necessary: float = 0.8
    beta_artificial: float = 0.36
    pw_smoothing: float = 0.5
    step_reduction_exp: float = 0.3
    step_growth_exp: float = 0.6
    stall_checks: int = 0
    # infeasibility detection (a reading; PDLP-style, the paper delegates the LP solve):
    # at each check the candidate ray is the unscaled y minus y at the last earlier check
    # whose index is a power of two, with the entries that would need an infinite row side
    # set to 0; the solve ends INFEASIBLE when D(candidate) > infeas_margin * S
    # (oracle/infeas.py), which weak duality rules out on a feasible LP
    infeasibility_checks: bool = False
    infeas_margin: float = 1e-9


def precondition(A: sp.csr_matrix, ruiz_iters: int, pock_chambolle: bool):
    """Row and column multipliers R, C with A~ = diag(R) A diag(C).

    Ruiz: each pass divides R_i by sqrt(max_j |A~_ij|) and C_j by
    sqrt(max_i |A~_ij|), both taken on the same A~.  Pock-Chambolle (alpha = 1):
    R_i /= sqrt(sum_j |A~_ij|), C_j /= sqrt(sum_i |A~_ij|).  A zero norm leaves the
    multiplier unchanged.
    """
    m, n = A.shape
    R = np.ones(m)
    C = np.ones(n)
    absA = abs(A).tocsr()
    for _ in range(ruiz_iters):
        S = sp.diags(R) @ absA @ sp.diags(C)
        rmax = np.asarray(S.max(axis=1).todense()).ravel() if m and n else np.zeros(m)
        cmax = np.asarray(S.max(axis=0).todense()).ravel() if m and n else np.zeros(n)
        R = R / np.sqrt(np.where(rmax > 0, rmax, 1.0))
        C = C / np.sqrt(np.where(cmax > 0, cmax, 1.0))
    if pock_chambolle:
        S = sp.diags(R) @ absA @ sp.diags(C)
        rsum = np.asarray(S.sum(axis=1)).ravel()
        csum = np.asarray(S.sum(axis=0)).ravel()
        R = R / np.sqrt(np.where(rsum > 0, rsum, 1.0))
        C = C / np.sqrt(np.where(csum > 0, csum, 1.0))
    return R, C


def bound_norm_vector(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Per row, the largest finite |lo_i|, |hi_i| (0 if both are infinite)."""
    a = np.where(np.isfinite(lo), np.abs(lo), 0.0)
    b = np.where(np.isfinite(hi), np.abs(hi), 0.0)
    return np.maximum(a, b)


def dual_prox(y, tau_y, Axt, lo, hi):
    """Dual step of Algorithm 1 generalised to row bounds (see module docstring)."""
    with np.errstate(invalid="ignore"):
        t_lo = y + tau_y * (lo - Axt)
        t_hi = y + tau_y * (hi - Axt)
    out = np.zeros_like(y)
    case_lo = np.isfinite(lo) & (t_lo > 0)
    case_hi = ~case_lo & np.isfinite(hi) & (t_hi < 0)
    out[case_lo] = t_lo[case_lo]
    out[case_hi] = t_hi[case_hi]
    return out


def reduced_cost_projection(r, l, u):
    """lambda = proj_Lambda(r): Lambda_j = R (both bounds finite), R+ (only l finite),
    R- (only u finite), {0} (free column)."""
    lf = np.isfinite(l)
    uf = np.isfinite(u)
    lam = np.where(lf & uf, r, np.where(lf, np.maximum(r, 0.0), np.where(uf, np.minimum(r, 0.0), 0.0)))
    return lam


def _splitmix64_finalize(z: np.ndarray) -> np.ndarray:
    # SplitMix64 output function (Steele, Lea, Flood 2014), on uint64 arrays
    z = z.astype(np.uint64)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def rounding_hash(x_int_cols: np.ndarray, cols: np.ndarray) -> int:
    """Order-independent 64-bit hash of round(x_j) over the given integer columns.

    Sum over j (mod 2^64) of mix(j * 0x9E3779B97F4A7C15 + r_j), r_j = floor(x_j + 1/2)
    clamped to +-2^62, mix = the SplitMix64 output function.
    """
    if len(cols) == 0:
        return 0
    r = np.floor(x_int_cols + 0.5)
    r = np.clip(r, -(2.0 ** 62), 2.0 ** 62).astype(np.int64).view(np.uint64)
    with np.errstate(over="ignore"):
        key = cols.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15) + r
        h = _splitmix64_finalize(key)
    return int(np.sum(h, dtype=np.uint64)) & MASK64


@dataclass
class Evaluation:
    eps_p: float
    eps_d: float
    eps_g: float
    rel_kkt: float
    pobj: float
    dobj: float
    rp_s2: float  # ||scaled primal residual||^2
    rd_s2: float  # ||scaled dual residual||^2

    def weighted_kkt(self, omega: float) -> float:
        g = self.pobj - self.dobj
        return math.sqrt(omega * omega * self.rp_s2 + self.rd_s2 / (omega * omega) + g * g)


@dataclass
class SolveResult:
    status: int
    iterations: int
    accepted: int
    rejected: int
    restarts: int
    eps_p: float
    eps_d: float
    eps_g: float
    rel_kkt: float
    pobj: float
    dobj: float
    used_average: bool
    trace: list = field(default_factory=list)
    certificate: "np.ndarray | None" = None  # the dual ray when status is INFEASIBLE


class OracleLP:
    """The LP ``min c^T x, lo <= Ax <= hi, l <= x <= u`` and its PDHG state.

    The constructor takes the LP exactly as the caller gives it (no auxiliary
    columns; ``oracle.pump.augment`` builds those).  ``int_cols`` lists the
    integer columns used by the stall test (Algorithm 1, "bounds stalling").
    """

    def __init__(self, A: sp.csr_matrix, c, lo, hi, l, u, int_cols=None, params: PdhgParams | None = None,
                 offset: float = 0.0, q=None):
        self.p = params or PdhgParams()
        self.A = sp.csr_matrix(A, dtype=np.float64)
        self.m, self.n = self.A.shape
        self.lo = np.asarray(lo, dtype=np.float64).copy()
        self.hi = np.asarray(hi, dtype=np.float64).copy()
        self.l = np.asarray(l, dtype=np.float64).copy()
        self.u = np.asarray(u, dtype=np.float64).copy()
        self.int_cols = np.asarray(int_cols if int_cols is not None else [], dtype=np.int64)
        self.R, self.C = precondition(self.A, self.p.ruiz_iters, self.p.pock_chambolle)
        self.As = (sp.diags(self.R) @ self.A @ sp.diags(self.C)).tocsr()
        self.AsT = self.As.T.tocsr()
        self.l_s = self.l / self.C
        self.u_s = self.u / self.C
        self._set_row_bounds(self.lo, self.hi)
        self.set_objective_vector(np.asarray(c, dtype=np.float64), offset)
        self.set_quadratic(q)
        # initial step size and primal weight (on the scaled LP)
        amax = float(np.max(np.abs(self.As.data))) if self.As.nnz else 0.0
        if self.p.adaptive_step:
            self.eta = 1.0 / amax if amax > 0 else 1.0
        else:
            fro = float(np.sqrt(np.sum(self.As.data ** 2)))
            self.eta = self.p.fixed_step_factor / fro if fro > 0 else 1.0
        cn = float(np.linalg.norm(self.c_s))
        qn = float(np.linalg.norm(bound_norm_vector(self.lo_s, self.hi_s)))
        self.omega = cn / qn if (cn > 0 and qn > 0) else 1.0
        self.x = np.clip(np.zeros(self.n), self.l_s, self.u_s)
        self.y = np.zeros(self.m)

    # -- data that changes between pump rounds ---------------------------------
    def _set_row_bounds(self, lo, hi):
        self.lo = np.asarray(lo, dtype=np.float64).copy()
        self.hi = np.asarray(hi, dtype=np.float64).copy()
        self.lo_s = self.lo * self.R
        self.hi_s = self.hi * self.R
        self.bnorm = float(np.linalg.norm(bound_norm_vector(self.lo, self.hi)))

    def set_row_bounds(self, lo, hi):
        self._set_row_bounds(lo, hi)

    def set_quadratic(self, q):
        """Diagonal of the objective's Hessian (unscaled, length n, >= 0); None for
        the LP."""
        self.has_q = q is not None
        self.q = np.zeros(self.n) if q is None else np.asarray(q, dtype=np.float64).copy()
        self.q_s = self.q * self.C * self.C

    def set_objective_vector(self, c, offset: float = 0.0):
        self.c = np.asarray(c, dtype=np.float64).copy()
        self.offset = float(offset)
        self.c_s = self.c * self.C
        self.cnorm = float(np.linalg.norm(self.c))

    # -- unscaled views of the state -------------------------------------------
    def primal(self, x_s=None):
        return (self.x if x_s is None else x_s) * self.C

    def dual(self, y_s=None):
        return (self.y if y_s is None else y_s) * self.R

    def set_state(self, x, y):
        """Set the iterate from unscaled x, y."""
        self.x = np.asarray(x, dtype=np.float64) / self.C
        self.y = np.asarray(y, dtype=np.float64) / self.R

    # -- Section 2.2: residuals and gap ----------------------------------------
    def evaluate(self, x, y) -> Evaluation:
        """Relative KKT error of a scaled iterate, measured on the original LP.

        eps_p = ||Ax - proj_[lo,hi](Ax)||_2 / (1 + ||b||_2), b_i the largest finite
        |lo_i|, |hi_i|; eps_d = ||r - lambda||_2 / (1 + ||c||_2) with r = c - A^T y
        and lambda its projection onto the sign cone of the column bounds;
        eps_g = |p - d| / (1 + |p| + |d|), where d takes lo_i y_i for y_i > 0, hi_i y_i
        for y_i < 0 and the same with l, u and lambda.  A y_i whose sign needs an
        infinite row side makes d = -inf; PDHG iterates never have one, because the
        dual step keeps every y_i in the sign cone of its row's finite sides.
        """
        Ax = self.As @ x
        ATy = self.AsT @ y
        rps = Ax - np.clip(Ax, self.lo_s, self.hi_s)
        qx = self.q_s * x if self.has_q else None
        r = (self.c_s + qx - ATy) if self.has_q else (self.c_s - ATy)
        lam = reduced_cost_projection(r, self.l_s, self.u_s)
        rds = r - lam
        xqx = 0.5 * float(x @ qx) if self.has_q else 0.0
        pobj = float(self.c_s @ x) + xqx + self.offset
        yp = np.maximum(y, 0.0)
        yn = np.maximum(-y, 0.0)
        lp = np.maximum(lam, 0.0)
        ln_ = np.maximum(-lam, 0.0)
        with np.errstate(invalid="ignore"):
            row_terms = np.where(yp > 0, self.lo_s * yp, 0.0) - np.where(yn > 0, self.hi_s * yn, 0.0)
            col_terms = np.where(lp > 0, self.l_s * lp, 0.0) - np.where(ln_ > 0, self.u_s * ln_, 0.0)
        dobj = float(np.sum(row_terms)) + float(np.sum(col_terms)) - xqx + self.offset
        rp = rps / self.R
        rd = rds / self.C
        eps_p = float(np.linalg.norm(rp)) / (1.0 + self.bnorm)
        eps_d = float(np.linalg.norm(rd)) / (1.0 + self.cnorm)
        eps_g = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
        return Evaluation(eps_p, eps_d, eps_g, max(eps_p, eps_d, eps_g), pobj, dobj,
                          float(rps @ rps), float(rds @ rds))

    # -- one PDHG step (Algorithm 1, inner loop body) ---------------------------
    def pdhg_step(self, x, y, eta, omega):
        tau_x = eta / omega
        tau_y = eta * omega
        d_x = self.AsT @ y - self.c_s
        v = x + tau_x * d_x
        if self.has_q:
            v = v / (1.0 + tau_x * self.q_s)
        x_new = np.clip(v, self.l_s, self.u_s)
        Axt = self.As @ (2.0 * x_new - x)
        y_new = dual_prox(y, tau_y, Axt, self.lo_s, self.hi_s)
        return x_new, y_new

    def primal_step_at(self, cols, x, y, eta, omega):
        """x'_j of one PDHG step for the listed columns only (sampled parity)."""
        cols = np.asarray(cols)
        tau_x = eta / omega
        sub = self.As[:, cols].tocsc()
        d_x = sub.T @ y - self.c_s[cols]
        v = x[cols] + tau_x * d_x
        if self.has_q:
            v = v / (1.0 + tau_x * self.q_s[cols])
        return np.clip(v, self.l_s[cols], self.u_s[cols])

    def dual_step_at(self, rows, x, x_new, y, eta, omega):
        """y'_i of one PDHG step for the listed rows only (sampled parity)."""
        rows = np.asarray(rows)
        tau_y = eta * omega
        Axt = self.As[rows, :] @ (2.0 * x_new - x)
        return dual_prox(y[rows], tau_y, Axt, self.lo_s[rows], self.hi_s[rows])

    def stall_hash(self, x_s) -> int:
        ic = self.int_cols
        return rounding_hash((x_s[ic] * self.C[ic]) if len(ic) else np.zeros(0), ic)

    # -- Algorithm 1 inner loop with PDLP's step size, averaging and restarts ---
    def solve(self, tol: float, iter_limit: int, trace: bool = False, replay=None) -> SolveResult:
        """PDHG from the current pair until rel-KKT <= tol or k = iter_limit.

        ``trace`` records, per attempt, ("step", k, accept, eta_used, eta_max,
        eta_next, cond, step_cond) and, per check that neither starts nor ends the solve,
        ("check", k, restart, candidate_is_average, omega_after, kkt_candidate,
        restart_margin, candidate_margin, omega_cond) -- all as this oracle computes
        them.  ``cond`` is the condition number of the interaction term
        sum_i |dy_i| (|A| (|x'| + |x|))_i / |dy.A dx| (how much a rounding of A x'
        or A x moves it) and ``step_cond`` is ||z|| / ||z' - z|| (how much a relative
        change of the iterate moves the step); the margins are the relative distances of the candidate's
        weighted KKT to the restart thresholds and to the other candidate's;
        ``omega_cond`` is (||x_c|| / ||x_c - x_lr|| + ||y_c|| / ||y_c - y_lr||).  ``replay = (steps, checks)`` takes the
        scalar decisions from another implementation's trace instead (eta used,
        accept, eta next per attempt; restart, candidate and omega per check) while
        still computing and recording its own: adaptive PDHG amplifies rounding
        differences chaotically, so iterate parity beyond a few attempts is only
        meaningful along the same decision sequence.
        """
        p = self.p
        if replay is not None:
            trace = True
            r_steps, r_checks = replay
        ci = 0
        x, y = self.x, self.y
        eta, omega = self.eta, self.omega
        k = 0
        accepted = rejected = restarts = 0
        wsum = 0.0
        x_avg = np.zeros(self.n)
        y_avg = np.zeros(self.m)
        tr = []

        ev_c = self.evaluate(x, y)
        x_lr, y_lr, k_lr = x, y, 0
        kkt_lr = ev_c.weighted_kkt(omega)
        kkt_prev = kkt_lr
        last_hash = self.stall_hash(x)
        same_hash = 0
        y_anchor = None
        certificate = None
        status = None
        out = (x, y, ev_c, False)
        if ev_c.rel_kkt <= tol:
            status = CONVERGED
        while status is None and k < iter_limit:
            if replay is not None:
                eta = float(r_steps[k][0])
            x_new, y_new = self.pdhg_step(x, y, eta, omega)
            eta_max = INF
            cond = 0.0
            step_cond = 0.0
            if p.adaptive_step:
                dx = x_new - x
                dy = y_new - y
                interaction = float(dy @ (self.As @ dx))
                if trace:
                    # diagnostics of the trace only (no effect on the iterates)
                    absA = abs(self.As)
                    scale = float(np.abs(dy) @ (absA @ (np.abs(x_new) + np.abs(x))))
                    cond = scale / abs(interaction) if interaction != 0.0 else INF
                    dz = math.sqrt(float(dx @ dx) + float(dy @ dy))
                    zn = math.sqrt(float(x @ x) + float(y @ y))
                    step_cond = zn / dz if dz > 0 else INF
                movement = omega * float(dx @ dx) + float(dy @ dy) / omega
                eta_max = movement / (2.0 * abs(interaction)) if interaction != 0.0 else INF
                kk = k + 2  # (k+1) with k the 1-based number of this attempt
                eta_next = min((1.0 - kk ** (-p.step_reduction_exp)) * eta_max,
                               (1.0 + kk ** (-p.step_growth_exp)) * eta)
                accept = eta <= eta_max
                eta_used = eta
                eta = eta_next
            else:
                accept = True
                eta_used = eta
            k += 1
            if trace:
                tr.append(("step", k, bool(accept), eta_used, eta_max, eta, cond, step_cond))
            if replay is not None:
                accept = bool(r_steps[k - 1][2] > 0.5)
                eta = float(r_steps[k - 1][3])
            if accept:
                accepted += 1
                x, y = x_new, y_new
                wsum += eta_used
                w = eta_used / wsum
                x_avg = (1.0 - w) * x_avg + w * x
                y_avg = (1.0 - w) * y_avg + w * y
            else:
                rejected += 1
            if k % p.n_check != 0 and k != iter_limit:
                continue
            # -- check: termination (Section 2.2), stalling, restart ----------
            ev_c = self.evaluate(x, y)
            ev_a = self.evaluate(x_avg, y_avg) if wsum > 0 else None
            if ev_a is not None and ev_a.rel_kkt < ev_c.rel_kkt:
                out = (x_avg, y_avg, ev_a, True)
            else:
                out = (x, y, ev_c, False)
            if out[2].rel_kkt <= tol:
                status = CONVERGED
                break
            if k >= iter_limit:
                status = ITER_LIMIT
                break
            h = self.stall_hash(x)
            same_hash = same_hash + 1 if h == last_hash else 0
            last_hash = h
            if p.stall_checks > 0 and same_hash >= p.stall_checks:
                status = STALLED
                break
            if p.infeasibility_checks:
                n_chk = k // p.n_check
                yu = self.dual(y)
                if y_anchor is not None:
                    cand = infeas.sign_projection(yu - y_anchor, self.lo, self.hi)
                    g, sc = infeas.farkas_gap_scale(self.A, self.lo, self.hi, self.l, self.u, cand)
                    if g > p.infeas_margin * sc:
                        certificate = cand
                        status = INFEASIBLE
                        break
                if n_chk & (n_chk - 1) == 0:
                    y_anchor = yu
            if not p.restarts:
                continue
            kc_cur = ev_c.weighted_kkt(omega)
            if ev_a is not None and ev_a.weighted_kkt(omega) < kc_cur:
                xc, yc, evc, is_avg = x_avg, y_avg, ev_a, True
            else:
                xc, yc, evc, is_avg = x, y, ev_c, False
            kc = evc.weighted_kkt(omega)
            other = ev_c if is_avg else ev_a
            cand_margin = (abs(other.weighted_kkt(omega) - kc) / kc) if (other is not None and kc > 0) else INF
            thresholds = [p.beta_sufficient * kkt_lr, p.beta_necessary * kkt_lr, kkt_prev]
            restart_margin = min(abs(kc - t) / kc for t in thresholds) if kc > 0 else INF
            do_restart = (kc <= p.beta_sufficient * kkt_lr
                          or (kc <= p.beta_necessary * kkt_lr and kc > kkt_prev)
                          or (k - k_lr) >= p.beta_artificial * k)
            omega_new = omega
            omega_cond = 0.0
            if do_restart and p.primal_weight_update:
                ddx = float(np.linalg.norm(xc - x_lr))
                ddy = float(np.linalg.norm(yc - y_lr))
                if ddx > 1e-10 and ddy > 1e-10:
                    omega_cond = float(np.linalg.norm(xc)) / ddx + float(np.linalg.norm(yc)) / ddy
                    omega_new = math.exp(p.pw_smoothing * math.log(ddy / ddx)
                                         + (1.0 - p.pw_smoothing) * math.log(omega))
            if trace:
                tr.append(("check", k, bool(do_restart), is_avg, omega_new, kc, restart_margin, cand_margin,
                           omega_cond))
            if replay is not None:
                rec = r_checks[ci]
                ci += 1
                do_restart = bool(rec[1] > 0.5)
                is_avg = bool(rec[2] > 0.5)
                xc, yc, evc = (x_avg, y_avg, ev_a) if is_avg else (x, y, ev_c)
                omega_new = float(rec[3])
            if do_restart:
                restarts += 1
                omega = omega_new
                x, y = xc, yc
                x_lr, y_lr, k_lr = xc, yc, k
                wsum = 0.0
                kkt_lr = evc.weighted_kkt(omega)
                kkt_prev = kkt_lr
            else:
                kkt_prev = kc
        if status is None:
            status = ITER_LIMIT
        xo, yo, evo, used_avg = out
        self.x, self.y = xo, yo
        self.eta, self.omega = eta, omega
        return SolveResult(status, k, accepted, rejected, restarts, evo.eps_p, evo.eps_d, evo.eps_g,
                           evo.rel_kkt, evo.pobj, evo.dobj, used_avg, tr, certificate)
