"""The C ABI library loads, exports every symbol the header declares, agrees with
the binding's struct layouts, and rejects malformed input before touching a GPU."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2307_03466_gb300 import build as B
from paper_2307_03466_gb300 import scylla as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "scylla.h")


@pytest.fixture(scope="module")
def L():
    B.build()
    return S.lib()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(scylla_\w+)\s*\(", txt)))


def test_header_and_binding_agree(L):
    decl = declared_functions()
    assert decl, "no declarations parsed"
    assert sorted(S.exported_symbols()) == decl


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", S.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_struct_layout_matches_c_compiler(L):
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "scylla.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(scylla_csr), sizeof(scylla_params), sizeof(scylla_pdhg_result),
         sizeof(scylla_run_result), sizeof(scylla_repair_result));
  printf("%zu %zu %zu %zu %zu\n", offsetof(scylla_params, fixed_step_factor), offsetof(scylla_params, seed),
         offsetof(scylla_params, time_limit_s), offsetof(scylla_params, repair_iters),
         offsetof(scylla_params, repair_tol));
  printf("%zu %zu %zu %zu %zu\n", offsetof(scylla_params, repair_rounds), offsetof(scylla_repair_result, rel_kkt),
         offsetof(scylla_params, distance), offsetof(scylla_params, batch_launch), offsetof(scylla_params, autotune));
  printf("%zu %zu %zu\n", offsetof(scylla_params, infeasibility_checks), offsetof(scylla_params, dual_form),
         offsetof(scylla_pdhg_result, kernel_form_dual));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "t.c")
        open(p, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), p, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[:5] == [C.sizeof(S.Csr), C.sizeof(S.Params), C.sizeof(S.PdhgResult), C.sizeof(S.RunResult),
                         C.sizeof(S.RepairResult)]
    assert sizes[5:] == [S.Params.fixed_step_factor.offset, S.Params.seed.offset, S.Params.time_limit_s.offset,
                         S.Params.repair_iters.offset, S.Params.repair_tol.offset,
                         S.Params.repair_rounds.offset, S.RepairResult.rel_kkt.offset, S.Params.distance.offset,
                         S.Params.batch_launch.offset, S.Params.autotune.offset,
                         S.Params.infeasibility_checks.offset, S.Params.dual_form.offset,
                         S.PdhgResult.kernel_form_dual.offset]


def test_default_params_are_the_papers(L):
    p = S.default_params()
    # Algorithm 1 (alpha) and Section 2.2 (eps1, beta, floor)
    assert (p.alpha, p.eps1, p.beta, p.eps_floor) == (0.9, 0.01, 0.98, 1e-8)
    assert p.n_check == 64 and p.precision == S.PREC_FP64
    # the continuous repair is not part of Algorithm 1: off unless asked for
    assert p.repair_iters == 0 and p.repair_tol == 1e-7 and p.repair_rounds == 8
    assert p.distance == 1  # Algorithm 1's l1 distance
    assert p.infeasibility_checks == 0  # the detector is a reading of the LP solver's, off by default


def _create(rowptr, cols, vals, m, n, lo=None, hi=None, l=None, u=None, c=None, ii=None):
    return S.LP(rowptr, cols, vals, np.zeros(n) if c is None else c,
                np.full(m, 1.0) if lo is None else lo, np.full(m, np.inf) if hi is None else hi,
                np.zeros(n) if l is None else l, np.ones(n) if u is None else u,
                np.zeros(n, np.uint8) if ii is None else ii, m, n)


@pytest.mark.parametrize("case,needle", [
    (dict(rowptr=[0, 2], cols=[1, 0], vals=[1.0, 1.0], m=1, n=2), "strictly increasing"),
    (dict(rowptr=[0, 2], cols=[0, 0], vals=[1.0, 1.0], m=1, n=2), "strictly increasing"),
    (dict(rowptr=[0, 1], cols=[5], vals=[1.0], m=1, n=2), "out of range"),
    (dict(rowptr=[0, 1], cols=[0], vals=[np.nan], m=1, n=2), "non-finite"),
    (dict(rowptr=[1, 1], cols=[], vals=[], m=1, n=2), "rowptr"),
    # rowptr[m] beyond the arrays: the binding passes their length as nnz, so the
    # library reports it instead of reading past them
    (dict(rowptr=[0, 2], cols=[0], vals=[1.0], m=1, n=2), "rowptr"),
    (dict(rowptr=[0, 1], cols=[0], vals=[1.0], m=1, n=2, lo=[2.0], hi=[1.0]), "row bounds"),
    (dict(rowptr=[0, 1], cols=[0], vals=[1.0], m=1, n=2, l=[0.0, 2.0], u=[1.0, 1.0]), "column bounds"),
    (dict(rowptr=[0, 1], cols=[0], vals=[1.0], m=1, n=2, c=[np.inf, 0.0]), "objective"),
    (dict(rowptr=[0, 1], cols=[0], vals=[1.0], m=1, n=2, ii=[1, 0], u=[1.5, 1.0]), "fractional"),
    (dict(rowptr=[0, 1], cols=[0], vals=[1.0], m=1, n=2, ii=[2, 0]), "0 or 1"),
])
def test_invalid_input_rejected_without_gpu(L, case, needle):
    with pytest.raises(S.ScyllaError) as ei:
        _create(**case)
    assert ei.value.code == S.ERR_INVALID_ARG
    assert needle in str(ei.value)


@pytest.mark.parametrize("case,needle", [
    (dict(rowptr=[0, 1], cols=[0], vals=[1.0], m=2, n=2, lo=[1.0, 1.0], hi=[2.0, 2.0]), "rowptr"),
    (dict(rowptr=[0, 1, 2], cols=[0], vals=[1.0], m=1, n=2), "rowptr"),
    (dict(rowptr=[0, 2], cols=[0, 1], vals=[1.0], m=1, n=2), "cols and vals"),
    (dict(rowptr=[0, 1], cols=[0], vals=[1.0], m=1, n=2, ii=[0, 0, 0]), "is_integer"),
])
def test_binding_checks_array_lengths_before_the_library(L, case, needle):
    """Lengths the C ABI cannot see (it takes plain pointers) are checked by the binding."""
    with pytest.raises(ValueError) as ei:
        _create(**case)
    assert needle in str(ei.value)


def test_binding_passes_the_first_nnz_entries_of_longer_arrays(L):
    """scipy CSR arrays may hold spare capacity beyond rowptr[m]: only the first nnz
    entries reach the library (here the spare entry would be out of range)."""
    with pytest.raises(S.ScyllaError) as ei:
        _create(rowptr=[0, 1], cols=[0, 9], vals=[1.0, 1.0], m=1, n=2, lo=[2.0], hi=[1.0])
    assert "row bounds" in str(ei.value)  # got past the CSR checks to the bounds
    rp, ci, va, nnz = S._csr([0, 1], [0, 9], [1.0, 1.0], 1)
    assert nnz == 1 and list(ci) == [0] and list(va) == [1.0]


def test_fanout_targets_shape_checked_by_the_binding(L):
    import types
    with pytest.raises(ValueError):
        S.Fanout(types.SimpleNamespace(n=5, h=None), np.zeros(5))
    with pytest.raises(ValueError):
        S.Fanout(types.SimpleNamespace(n=5, h=None), np.zeros((4, 3)))


def test_new_binding_methods_marshal_through_ctypes(L):
    """The batched fix-and-propagate and the certificate test: shapes checked in
    Python, then a null handle comes back from the library as INVALID_ARG (so the
    argument lists match the C signatures)."""
    import types
    fake = types.SimpleNamespace(n=5, m=3, h=None)
    with pytest.raises(ValueError):
        S.LP.fix_and_propagate_many(fake, np.zeros((2, 4)))
    with pytest.raises(S.ScyllaError) as ei:
        S.LP.fix_and_propagate_many(fake, np.zeros((2, 5)))
    assert ei.value.code == S.ERR_INVALID_ARG
    with pytest.raises(S.ScyllaError) as ei:
        S.LP.farkas_gap(fake, np.zeros(3))
    assert ei.value.code == S.ERR_INVALID_ARG


def test_null_handle_calls_fail_cleanly(L):
    r = S.PdhgResult()
    assert L.scylla_pdhg_solve(None, 1e-4, 10, C.byref(r)) == S.ERR_INVALID_ARG
    assert L.scylla_set_objective(None, None, 1) == S.ERR_INVALID_ARG
    assert L.scylla_set_col_bounds(None, None, None) == S.ERR_INVALID_ARG
    assert L.scylla_set_row_bounds(None, None, None) == S.ERR_INVALID_ARG
    assert L.scylla_set_qp_objective(None, None, None, 0.0) == S.ERR_INVALID_ARG
    assert L.scylla_propagate(None, None, None, None, 10, None, None) == S.ERR_INVALID_ARG
    rr = S.RepairResult()
    assert L.scylla_repair(None, None, 1e-6, 10, None, C.byref(rr)) == S.ERR_INVALID_ARG
    L.scylla_lp_destroy(None)
    assert b"null" in L.scylla_last_error()


def test_product_path_has_no_oracle_import():
    """The CUDA path's package never imports the oracle (it only exists for tests)."""
    pkg = os.path.join(ROOT, "paper_2307_03466_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                txt = open(os.path.join(dp, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
