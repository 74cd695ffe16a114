"""Thin Python binding of the C ABI in ``include/scylla.h`` (ctypes).

Argument marshalling only: every step of the PDHG path runs in the CUDA kernels of
``libscylla.so`` and the host rounding step in its C++ code.  The names follow the
C functions (``scylla_lp_create`` -> ``LP(...)``, ``scylla_pdhg_solve`` ->
``LP.pdhg_solve`` ...).  If the library is missing this module raises at import
of ``lib()``: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libscylla.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -6
CONVERGED, ITER_LIMIT, STALLED, NUMERICAL, DEVICE_TIMEOUT, INFEASIBLE = 0, 1, 2, 3, 4, 5
FOUND, NOT_FOUND = 0, 1
PREC_FP64, PREC_MIXED = 0, 1


class ScyllaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"scylla error {code}: {msg}")
        self.code = code


class Csr(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64),
                ("rowptr", C.POINTER(C.c_int64)), ("cols", C.POINTER(C.c_int32)),
                ("vals", C.POINTER(C.c_double))]


class Params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("n_check", C.c_int32), ("ruiz_iters", C.c_int32),
                ("pock_chambolle", C.c_int32), ("adaptive_step", C.c_int32), ("restarts", C.c_int32),
                ("primal_weight_update", C.c_int32), ("stall_checks", C.c_int32),
                ("aux_general_integers", C.c_int32), ("use_graph", C.c_int32),
                ("fixed_step_factor", C.c_double), ("beta_sufficient", C.c_double),
                ("beta_necessary", C.c_double), ("beta_artificial", C.c_double), ("pw_smoothing", C.c_double),
                ("step_reduction_exp", C.c_double), ("step_growth_exp", C.c_double),
                ("alpha", C.c_double), ("eps1", C.c_double), ("beta", C.c_double), ("eps_floor", C.c_double),
                ("max_rounds", C.c_int64), ("iter_limit", C.c_int64), ("total_iter_cap", C.c_int64),
                ("run_stall_checks", C.c_int32), ("trace_capacity", C.c_int32), ("seed", C.c_uint64),
                ("time_limit_s", C.c_double), ("device_wait_limit_s", C.c_double), ("pdl", C.c_int32),
                ("prefetch", C.c_int32), ("host_transpose", C.c_int32),
                ("repair_iters", C.c_int64), ("repair_tol", C.c_double), ("repair_rounds", C.c_int32),
                ("distance", C.c_int32), ("batch_launch", C.c_int32), ("autotune", C.c_int32),
                ("infeasibility_checks", C.c_int32), ("dual_form", C.c_int32)]


class PdhgResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("used_average", C.c_int32), ("iterations", C.c_int64),
                ("accepted", C.c_int64), ("rejected", C.c_int64), ("restarts", C.c_int64),
                ("eps_p", C.c_double), ("eps_d", C.c_double), ("eps_g", C.c_double), ("rel_kkt", C.c_double),
                ("pobj", C.c_double), ("dobj", C.c_double), ("eta", C.c_double), ("omega", C.c_double),
                ("seconds", C.c_double), ("launches", C.c_int64), ("kernel_form", C.c_int32),
                ("kernel_form_dual", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RunResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("found_by", C.c_int32), ("rounds", C.c_int64),
                ("total_iterations", C.c_int64), ("perturbations", C.c_int64), ("objective", C.c_double),
                ("seconds", C.c_double), ("seconds_pdhg", C.c_double), ("seconds_fixprop", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RepairResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("pdhg_status", C.c_int32), ("iterations", C.c_int64),
                ("rounds", C.c_int32), ("shifted_rows", C.c_int32),
                ("rel_kkt", C.c_double), ("objective", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "scylla_default_params": (None, [C.POINTER(Params)]),
    "scylla_lp_create": (C.c_int, [C.POINTER(Csr), _D, _D, _D, _D, _D, C.POINTER(C.c_uint8),
                                   C.POINTER(Params), _P, C.POINTER(_P)]),
    "scylla_lp_destroy": (None, [_P]),
    "scylla_lp_dims": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64)]),
    "scylla_pdhg_solve": (C.c_int, [_P, C.c_double, C.c_int64, C.POINTER(PdhgResult)]),
    "scylla_set_objective": (C.c_int, [_P, _D, C.c_int32]),
    "scylla_get_objective": (C.c_int, [_P, _D, _D]),
    "scylla_set_qp_objective": (C.c_int, [_P, _D, _D, C.c_double]),
    "scylla_run": (C.c_int, [_P, _D, C.POINTER(RunResult)]),
    "scylla_get_primal": (C.c_int, [_P, _D]),
    "scylla_get_dual": (C.c_int, [_P, _D]),
    "scylla_get_primal_device": (C.c_int, [_P, C.c_void_p]),
    "scylla_get_state": (C.c_int, [_P, _D, _D, _D, _D]),
    "scylla_set_state": (C.c_int, [_P, _D, _D, C.c_double, C.c_double]),
    "scylla_get_scaling": (C.c_int, [_P, _D, _D]),
    "scylla_get_transpose": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int32), _D]),
    "scylla_fix_and_propagate": (C.c_int, [_P, _D, _D, _D, _D, C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                           C.POINTER(C.c_uint8)]),
    "scylla_check_feasible": (C.c_int, [_P, _D, C.POINTER(C.c_int32)]),
    "scylla_farkas_gap": (C.c_int, [_P, _D, _D]),
    "scylla_get_certificate": (C.c_int, [_P, _D, _D, _D]),
    "scylla_fix_and_propagate_many": (C.c_int, [_P, C.c_int32, _D, _D, _D, _D, C.POINTER(C.c_int64)]),
    "scylla_set_col_bounds": (C.c_int, [_P, _D, _D]),
    "scylla_set_row_bounds": (C.c_int, [_P, _D, _D]),
    "scylla_propagate": (C.c_int, [_P, _D, _D, C.POINTER(C.c_uint8), C.c_int64, C.POINTER(C.c_int64),
                                   C.POINTER(C.c_int64)]),
    "scylla_repair": (C.c_int, [_P, _D, C.c_double, C.c_int64, _D, C.POINTER(RepairResult)]),
    "scylla_perturb": (C.c_int, [_P, _D, _D, C.c_int32, C.c_int64, C.c_uint64, C.POINTER(C.c_int64)]),
    "scylla_get_trace": (C.c_int, [_P, _D, C.POINTER(C.c_int64), _D, C.POINTER(C.c_int64)]),
    "scylla_reset_state": (C.c_int, [_P]),
    "scylla_time_kernels": (C.c_int, [_P, C.c_int32, _D]),
    "scylla_kernel_form": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32), _D]),
    "scylla_primal_residual_noalloc": (C.c_int, [C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P]),
    "scylla_batch_create": (C.c_int, [C.c_int32, C.POINTER(Csr), C.POINTER(_D), C.POINTER(_D), C.POINTER(_D),
                                      C.POINTER(_D), C.POINTER(_D), C.POINTER(Params), _P, C.POINTER(_P)]),
    "scylla_batch_destroy": (None, [_P]),
    "scylla_batch_solve": (C.c_int, [_P, C.c_double, C.c_int64, C.POINTER(PdhgResult), _D]),
    "scylla_batch_get_primal": (C.c_int, [_P, C.c_int32, _D]),
    "scylla_batch_get_dual": (C.c_int, [_P, C.c_int32, _D]),
    "scylla_batch_reset_state": (C.c_int, [_P]),
    "scylla_fanout_create": (C.c_int, [_P, C.c_int32, _D, C.c_int32, C.POINTER(_P)]),
    "scylla_fanout_destroy": (None, [_P]),
    "scylla_fanout_solve": (C.c_int, [_P, C.c_double, C.c_int64, C.POINTER(PdhgResult), _D]),
    "scylla_fanout_get_primal": (C.c_int, [_P, C.c_int32, _D]),
    "scylla_fanout_get_dual": (C.c_int, [_P, C.c_int32, _D]),
    "scylla_fanout_reset_state": (C.c_int, [_P]),
    "scylla_batch_info": (C.c_int, [_P, C.POINTER(C.c_int32), _D]),
    "scylla_batch_time_kernels": (C.c_int, [_P, C.c_int32, _D]),
    "scylla_fanout_time_kernels": (C.c_int, [_P, C.c_int32, _D]),
    "scylla_fanout_tune": (C.c_int, [_P, C.c_int32, C.c_int32]),
    "scylla_fanout_info": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _D]),
    "scylla_last_error": (C.c_char_p, []),
}

_lib = None


def lib(path: str = LIB_PATH) -> C.CDLL:
    """Load libscylla.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} not built; run python -m paper_2307_03466_gb300.build")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc: int):
    if rc != OK:
        raise ScyllaError(rc, lib().scylla_last_error().decode())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def default_params(**kw) -> Params:
    p = Params()
    lib().scylla_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def primal_residual_noalloc(m: int, rowptr: int, cols: int, vals: int, x: int, row_lo: int, row_hi: int,
                            out: int, stream=None):
    """scylla_primal_residual_noalloc on caller-owned device pointers (ints); see the header."""
    _check(lib().scylla_primal_residual_noalloc(int(m), _P(rowptr), _P(cols), _P(vals), _P(x), _P(row_lo),
                                                 _P(row_hi), _P(out), _P(stream) if stream else None))


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (n,):
        raise ValueError(f"expected length {n}, got {a.shape}")
    return a


def _csr(rowptr, cols, vals, m: int):
    """The CSR arrays as the C ABI reads them.  The library gets plain pointers, so the
    lengths it cannot see are checked here: rowptr has m + 1 entries, and cols and vals
    have one length.  nnz is rowptr[m] when the arrays hold that many entries (longer
    arrays, such as scipy's with spare capacity, pass their first nnz entries), else the
    arrays' length, which the library then reports as inconsistent with rowptr[m]
    before it reads cols or vals."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    if m >= 0 and rp.shape != (m + 1,):
        raise ValueError(f"rowptr: expected length m + 1 = {m + 1}, got {rp.shape}")
    ci = np.ascontiguousarray(cols, dtype=np.int32)
    va = np.ascontiguousarray(vals, dtype=np.float64)
    if ci.ndim != 1 or ci.shape != va.shape:
        raise ValueError(f"cols and vals: expected two arrays of one length, got {ci.shape} and {va.shape}")
    nnz = int(rp[-1]) if rp.size else 0
    if 0 <= nnz <= ci.shape[0]:
        return rp, ci[:nnz], va[:nnz], nnz
    return rp, ci, va, int(ci.shape[0])


class LP:
    """An LP handle (``scylla_lp``).  Inputs are host arrays, copied at create."""

    def __init__(self, rowptr, cols, vals, c, row_lo, row_hi, col_lo, col_hi, is_integer, m: int, n: int,
                 params: Params | None = None, stream=None):
        L = lib()
        self.m, self.n = int(m), int(n)
        self._rowptr, self._cols, self._vals, nnz = _csr(rowptr, cols, vals, self.m)
        csr = Csr(self.m, self.n, nnz, self._rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                  self._cols.ctypes.data_as(C.POINTER(C.c_int32)), _dp(self._vals))
        c = _f64(c, n)
        lo = _f64(row_lo, m)
        hi = _f64(row_hi, m)
        l = _f64(col_lo, n)
        u = _f64(col_hi, n)
        ii = np.ascontiguousarray(is_integer, dtype=np.uint8)
        if ii.shape != (self.n,):
            raise ValueError(f"is_integer: expected length {self.n}, got {ii.shape}")
        self.params = params if params is not None else default_params()
        h = _P()
        st = _P(stream) if stream is not None else None
        _check(L.scylla_lp_create(C.byref(csr), _dp(c), _dp(lo), _dp(hi), _dp(l), _dp(u),
                                  ii.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(self.params), st, C.byref(h)))
        self.h = h
        mt, nt, zt, na = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        _check(L.scylla_lp_dims(self.h, C.byref(mt), C.byref(nt), C.byref(zt), C.byref(na)))
        self.m_total, self.n_total, self.nnz_total, self.n_aux = mt.value, nt.value, zt.value, na.value

    @classmethod
    def from_instance(cls, inst, params: Params | None = None, stream=None) -> "LP":
        return cls(inst.rowptr, inst.cols, inst.vals, inst.c, inst.lo, inst.hi, inst.l, inst.u, inst.is_int,
                   inst.m, inst.n, params, stream)

    def close(self):
        if getattr(self, "h", None):
            lib().scylla_lp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def pdhg_solve(self, tol: float, iter_limit: int) -> PdhgResult:
        r = PdhgResult()
        _check(lib().scylla_pdhg_solve(self.h, float(tol), int(iter_limit), C.byref(r)))
        return r

    def set_objective(self, xhat, K: int):
        x = _f64(xhat, self.n)
        _check(lib().scylla_set_objective(self.h, _dp(x), int(K)))

    def set_qp_objective(self, c, q, offset: float = 0.0):
        """min c^T x + 1/2 x^T diag(q) x + offset over the same constraints
        (scylla_set_qp_objective)."""
        cc = _f64(c, self.n)
        qq = _f64(q, self.n)
        _check(lib().scylla_set_qp_objective(self.h, _dp(cc), _dp(qq), float(offset)))

    def get_objective(self):
        c = np.empty(self.n_total)
        off = C.c_double()
        _check(lib().scylla_get_objective(self.h, _dp(c), C.byref(off)))
        return c, off.value

    def run(self):
        x = np.zeros(self.n)
        r = RunResult()
        _check(lib().scylla_run(self.h, _dp(x), C.byref(r)))
        return r, x

    def primal(self, out: "np.ndarray | None" = None) -> np.ndarray:
        """The primal iterate in the original space; written into ``out`` (a
        contiguous float64 array of length n) when given."""
        if out is None:
            x = np.empty(self.n)
        else:
            x = out
            if x.dtype != np.float64 or x.shape != (self.n,) or not x.flags["C_CONTIGUOUS"]:
                raise ValueError("out must be a contiguous float64 array of length n")
        _check(lib().scylla_get_primal(self.h, _dp(x)))
        return x

    def dual(self) -> np.ndarray:
        y = np.empty(self.m)
        _check(lib().scylla_get_dual(self.h, _dp(y) if self.m else None))
        return y

    def primal_device(self, ptr: int):
        _check(lib().scylla_get_primal_device(self.h, C.c_void_p(ptr)))

    def get_state(self):
        x = np.empty(self.n_total)
        y = np.empty(self.m_total)
        eta, om = C.c_double(), C.c_double()
        _check(lib().scylla_get_state(self.h, _dp(x), _dp(y) if self.m_total else None, C.byref(eta), C.byref(om)))
        return x, y, eta.value, om.value

    def set_state(self, x, y, eta: float, omega: float):
        x = _f64(x, self.n_total)
        y = _f64(y, self.m_total)
        _check(lib().scylla_set_state(self.h, _dp(x), _dp(y) if self.m_total else None, float(eta), float(omega)))

    def scaling(self):
        R = np.empty(self.m_total)
        Cc = np.empty(self.n_total)
        _check(lib().scylla_get_scaling(self.h, _dp(R) if self.m_total else None, _dp(Cc)))
        return R, Cc

    def transpose(self):
        """The stored transpose of the scaled matrix: (colptr, rows, vals)."""
        colptr = np.empty(self.n_total + 1, dtype=np.int64)
        _check(lib().scylla_get_transpose(self.h, colptr.ctypes.data_as(C.POINTER(C.c_int64)), None, None))
        nnz = int(colptr[-1])
        rows = np.empty(nnz, dtype=np.int32)
        vals = np.empty(nnz)
        _check(lib().scylla_get_transpose(self.h, None, rows.ctypes.data_as(C.POINTER(C.c_int32)), _dp(vals)))
        return colptr, rows, vals

    def fix_and_propagate(self, xbar):
        xb = _f64(xbar, self.n)
        xhat = np.empty(self.n)
        dl = np.empty(self.n)
        du = np.empty(self.n)
        fixed = np.empty(self.n, dtype=np.int32)
        nf = C.c_int64()
        ign = np.empty(max(self.m, 1), dtype=np.uint8)
        _check(lib().scylla_fix_and_propagate(self.h, _dp(xb), _dp(xhat), _dp(dl), _dp(du),
                                              fixed.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(nf),
                                              ign.ctypes.data_as(C.POINTER(C.c_uint8))))
        return xhat, dl, du, fixed[: nf.value].astype(np.int64), ign[: self.m].astype(bool)

    def fix_and_propagate_many(self, xbars):
        """Fix-and-propagate of K points at once on the host threads
        (scylla_fix_and_propagate_many): xbars of shape (K, n); returns xhat (K, n) and
        the number of columns fixed by rounding per point (K,)."""
        xb = np.ascontiguousarray(xbars, dtype=np.float64)
        if xb.ndim != 2 or xb.shape[1] != self.n:
            raise ValueError(f"xbars: expected shape (K, {self.n}), got {xb.shape}")
        K = xb.shape[0]
        xhat = np.empty((K, self.n))
        nf = np.zeros(K, dtype=np.int64)
        _check(lib().scylla_fix_and_propagate_many(self.h, int(K), _dp(xb), _dp(xhat), None, None,
                                                   nf.ctypes.data_as(C.POINTER(C.c_int64))))
        return xhat, nf

    def check_feasible(self, x) -> bool:
        xx = _f64(x, self.n)
        f = C.c_int32()
        _check(lib().scylla_check_feasible(self.h, _dp(xx), C.byref(f)))
        return bool(f.value)

    def farkas_gap(self, y) -> float:
        """D(y) of scylla_farkas_gap: > 0 proves the LP relaxation infeasible."""
        yy = _f64(y, self.m)
        g = C.c_double()
        _check(lib().scylla_farkas_gap(self.h, _dp(yy) if self.m else None, C.byref(g)))
        return g.value

    def certificate(self):
        """(y, gap, scale) of scylla_get_certificate: the dual ray tested at the last
        check of the last solve (unscaled, one entry per original row) and the D and S
        the device computed for it."""
        y = np.zeros(self.m)
        g, sc = C.c_double(), C.c_double()
        _check(lib().scylla_get_certificate(self.h, _dp(y) if self.m else None, C.byref(g), C.byref(sc)))
        return y, g.value, sc.value

    def reset_state(self):
        _check(lib().scylla_reset_state(self.h))

    def set_col_bounds(self, col_lo, col_hi):
        """New bounds of the original columns (scylla_set_col_bounds)."""
        lo = _f64(col_lo, self.n)
        hi = _f64(col_hi, self.n)
        _check(lib().scylla_set_col_bounds(self.h, _dp(lo), _dp(hi)))

    def propagate(self, dom_lo, dom_hi, max_rounds: int = 100000):
        """Bound propagation on the GPU (scylla_propagate): returns (dom_lo, dom_hi,
        ignored rows, rounds, conflicts)."""
        dl = _f64(dom_lo, self.n).copy()
        du = _f64(dom_hi, self.n).copy()
        ign = np.zeros(max(self.m, 1), dtype=np.uint8)
        rounds, conflicts = C.c_int64(), C.c_int64()
        _check(lib().scylla_propagate(self.h, _dp(dl), _dp(du), ign.ctypes.data_as(C.POINTER(C.c_uint8)),
                                      int(max_rounds), C.byref(rounds), C.byref(conflicts)))
        return dl, du, ign[: self.m].astype(bool), rounds.value, conflicts.value

    def set_row_bounds(self, row_lo, row_hi):
        """New bounds of the original rows (scylla_set_row_bounds)."""
        lo = _f64(row_lo, self.m)
        hi = _f64(row_hi, self.m)
        _check(lib().scylla_set_row_bounds(self.h, _dp(lo) if self.m else None, _dp(hi) if self.m else None))

    def repair(self, xhat, tol: float, iter_limit: int):
        """Continuous repair of xhat's integer assignment (scylla_repair): returns
        (RepairResult, x)."""
        xh = _f64(xhat, self.n)
        x = np.empty(self.n)
        r = RepairResult()
        _check(lib().scylla_repair(self.h, _dp(xh), float(tol), int(iter_limit), _dp(x), C.byref(r)))
        return r, x

    def kernel_form(self):
        """((primal form, dual form) in use, the L2-size rule's form, the autotuner's ms
        per launch: primal and dual of the 32-row form, of the wide form, of the
        asynchronous-copy form) -- scylla_kernel_form."""
        f, fd, r = C.c_int32(), C.c_int32(), C.c_int32()
        ms = np.zeros(6)
        _check(lib().scylla_kernel_form(self.h, C.byref(f), C.byref(fd), C.byref(r), _dp(ms)))
        return (f.value, fd.value), r.value, ms

    def time_kernels(self, attempts: int):
        """Mean device ms of (primal, dual, check-cols, check-rows) launches."""
        ms = np.zeros(4)
        _check(lib().scylla_time_kernels(self.h, int(attempts), _dp(ms)))
        return ms

    def trace(self):
        """(steps (N x 4), checks (M x 5)) of the last solve; see scylla_get_trace."""
        cap = int(self.params.trace_capacity)
        st = np.zeros(4 * max(cap, 1))
        ck = np.zeros(5 * max(cap, 1))
        ns, nc = C.c_int64(), C.c_int64()
        _check(lib().scylla_get_trace(self.h, _dp(st), C.byref(ns), _dp(ck), C.byref(nc)))
        return st[: 4 * ns.value].reshape(-1, 4), ck[: 5 * nc.value].reshape(-1, 5)

    def perturb(self, xhat, xbar, kind: int, K: int, seed: int):
        x = _f64(xhat, self.n).copy()
        xb = _f64(xbar, self.n)
        fl = C.c_int64()
        _check(lib().scylla_perturb(self.h, _dp(x), _dp(xb), int(kind), int(K), int(seed), C.byref(fl)))
        return x, fl.value


class Batch:
    """A batch of LP relaxations solved together (``scylla_batch``)."""

    def __init__(self, instances, params: Params | None = None, stream=None):
        L = lib()
        self.count = len(instances)
        keep = []
        csrs = (Csr * self.count)()
        arrs = {k: (_D * self.count)() for k in ("c", "lo", "hi", "l", "u")}
        self.sizes = []
        for b, inst in enumerate(instances):
            rp, ci, va, nnz = _csr(inst.rowptr, inst.cols, inst.vals, int(inst.m))
            keep += [rp, ci, va]
            csrs[b] = Csr(inst.m, inst.n, nnz, rp.ctypes.data_as(C.POINTER(C.c_int64)),
                          ci.ctypes.data_as(C.POINTER(C.c_int32)), _dp(va))
            for k, a, ln in (("c", inst.c, inst.n), ("lo", inst.lo, inst.m), ("hi", inst.hi, inst.m),
                             ("l", inst.l, inst.n), ("u", inst.u, inst.n)):
                v = _f64(a, ln)
                keep.append(v)
                arrs[k][b] = _dp(v)
            self.sizes.append((inst.m, inst.n))
        self.params = params if params is not None else default_params()
        h = _P()
        _check(L.scylla_batch_create(self.count, csrs, arrs["c"], arrs["lo"], arrs["hi"], arrs["l"], arrs["u"],
                                     C.byref(self.params), _P(stream) if stream else None, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().scylla_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, tol: float, iter_limit: int):
        res = (PdhgResult * self.count)()
        sec = C.c_double()
        _check(lib().scylla_batch_solve(self.h, float(tol), int(iter_limit), res, C.byref(sec)))
        return list(res), sec.value

    def primal(self, b: int) -> np.ndarray:
        x = np.empty(self.sizes[b][1])
        _check(lib().scylla_batch_get_primal(self.h, int(b), _dp(x)))
        return x

    def dual(self, b: int) -> np.ndarray:
        # an index out of range is the C call's error (INVALID_ARG)
        y = np.empty(self.sizes[b][0] if 0 <= b < len(self.sizes) else 1)
        _check(lib().scylla_batch_get_dual(self.h, int(b), _dp(y)))
        return y

    def reset_state(self):
        _check(lib().scylla_batch_reset_state(self.h))

    def info(self):
        """(the launch form in use: 1 graphs, 2 persistent work queue, 3 graphs over
        asynchronous-copy tiles; the create-time ms of n_check attempts in each form)."""
        p = C.c_int32()
        ms = np.zeros(3)
        _check(lib().scylla_batch_info(self.h, C.byref(p), _dp(ms)))
        return p.value, ms

    def time_kernels(self, attempts: int) -> np.ndarray:
        """Mean device ms of the primal step, dual step and step control of the graph
        form as separate launches (scylla_batch_time_kernels)."""
        ms = np.zeros(3)
        _check(lib().scylla_batch_time_kernels(self.h, int(attempts), _dp(ms)))
        return ms


class Fanout:
    """K pump objectives of one LP solved together (``scylla_fanout``).

    targets: array (n, K) of rounding targets; objective k is the Section 2.4 update
    of round ``round_K`` around column k.  The LP handle must outlive this object."""

    def __init__(self, lp: "LP", targets, round_K: int = 1):
        tg = np.asarray(targets, dtype=np.float64)
        if tg.ndim != 2 or tg.shape[0] != lp.n:
            raise ValueError(f"targets: expected shape (n, K) with n = {lp.n}, got {tg.shape}")
        t = np.ascontiguousarray(tg.T)  # K blocks of length n
        self.K = t.shape[0]
        self.lp = lp
        h = _P()
        _check(lib().scylla_fanout_create(lp.h, self.K, _dp(t), int(round_K), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().scylla_fanout_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, tol: float, iter_limit: int):
        res = (PdhgResult * self.K)()
        sec = C.c_double()
        _check(lib().scylla_fanout_solve(self.h, float(tol), int(iter_limit), res, C.byref(sec)))
        return list(res), sec.value

    def primal(self, k: int) -> np.ndarray:
        x = np.empty(self.lp.n)
        _check(lib().scylla_fanout_get_primal(self.h, int(k), _dp(x)))
        return x

    def dual(self, k: int) -> np.ndarray:
        y = np.empty(self.lp.m)
        _check(lib().scylla_fanout_get_dual(self.h, int(k), _dp(y)))
        return y

    def reset_state(self):
        _check(lib().scylla_fanout_reset_state(self.h))

    def tune(self, shape_primal: int = 0, shape_dual: int = 0):
        """scylla_fanout_tune: 0 times every tile shape, 1..4 forces one."""
        _check(lib().scylla_fanout_tune(self.h, int(shape_primal), int(shape_dual)))

    def info(self):
        """(tile shape of the primal and dual SpMM, the tuner's ms per launch: primal
        shapes 1..4, then dual shapes 1..4)."""
        a, b = C.c_int32(), C.c_int32()
        ms = np.zeros(8)
        _check(lib().scylla_fanout_info(self.h, C.byref(a), C.byref(b), _dp(ms)))
        return a.value, b.value, ms

    def time_kernels(self, attempts: int) -> np.ndarray:
        """Mean device ms of the primal SpMM, dual SpMM, step control, column check,
        row check and check control (scylla_fanout_time_kernels)."""
        ms = np.zeros(6)
        _check(lib().scylla_fanout_time_kernels(self.h, int(attempts), _dp(ms)))
        return ms
