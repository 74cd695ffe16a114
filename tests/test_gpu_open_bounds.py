"""GPU PDHG on LPs whose columns are not all boxed: lower-bounded only, upper-bounded
only, free and fixed columns, with covering, packing, two-sided, equality and free
rows (Algorithm 1's projection onto [l, u] with infinite sides; Section 2.2's
relative KKT error with the reduced-cost projection onto R+, R- and {0}).

The instances come from ``instances.open_bounds_lp`` and ``standard_form_lp``: LPs
built around a known optimal pair, so the converged objective has an exact value
beside the oracle's.  Parity is as in the other GPU tests: FP64 fixed-step iterates
within 1e-9 of the oracle, adaptive runs on the device's decisions, bit-identical
kernel forms on the same tiles, and FP32-mixed solves to 1e-4 re-evaluated by the
oracle, here with a dual residual that is not zero.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg as O
from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import TOL, TOL_LONG, compare_after, gpu_available, lib, pair, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# the oracle's own objective error at rel-KKT 1e-4 on these instances and on the
# mixed-precision tests' others is at most 8e-5; 1e-3 leaves a margin of ten
OBJ_TOL_MIXED = 1e-3


def _instances():
    return {
        "open_300x600": I.open_bounds_lp(300, 600, per_col=6, seed=31),
        "open_2kx4k": I.open_bounds_lp(2000, 4000, per_col=6, seed=21),
        # few nonzeros per column: transposed rows short, so the wide tiles hold > 32 rows
        "open_wide_3kx6k": I.open_bounds_lp(3000, 6000, per_col=3, seed=22),
        "standard_form_500x1500": I.standard_form_lp(500, 1500, per_col=5, seed=23),
    }


INSTANCES = _instances()


def test_device_evaluates_hand_example():
    """The check kernels' relative KKT error at the hand-worked non-optimal point
    (tests/golden/evaluate_nonoptimal.json): a zero-attempt solve evaluates the
    pair set on the handle, through the preconditioned LP, FP64 and FP32-mixed."""
    S = lib()
    d = json.load(open(os.path.join(GOLDEN, "evaluate_nonoptimal.json")))
    f = lambda v: np.array([float(t) for t in v])
    A = sp.csr_matrix(np.array(d["A_dense"], float))
    A.sort_indices()
    inst = I.Instance("hand", 3, 6, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.copy(),
                      f(d["c"]), f(d["row_lo"]), f(d["row_hi"]), f(d["col_lo"]), f(d["col_hi"]),
                      np.zeros(6, np.uint8))
    e = d["expected"]
    for prec, tol in ((0, 1e-14), (1, 1e-6)):
        g = S.LP.from_instance(inst, S.default_params(precision=prec, aux_general_integers=0))
        _, _, eta, omega = g.get_state()
        g.set_state(f(d["x"]), f(d["y"]), eta, omega)
        r = g.pdhg_solve(0.0, 0)
        assert abs(r.eps_p - e["eps_p_value"]) <= tol, (prec, r.eps_p)
        assert abs(r.eps_d - e["eps_d_value"]) <= tol, (prec, r.eps_d)
        assert abs(r.eps_g - e["eps_g_value"]) <= tol, (prec, r.eps_g)
        assert abs(r.pobj - e["pobj"]) <= tol * 10 and abs(r.dobj - e["dobj"]) <= tol * 10, (prec, r.pobj, r.dobj)
        g.close()


@pytest.mark.parametrize("name", list(INSTANCES))
def test_initial_point_and_preconditioning(name):
    """x = proj_[l,u](0) with infinite sides (Algorithm 1 initialisation, read as
    the projection of 0), y = 0, and the oracle's scaling."""
    inst = INSTANCES[name]
    g, o = pair(inst)
    R, C = g.scaling()
    assert rel_err(R, o.R) <= 1e-13 and rel_err(C, o.C) <= 1e-13
    x, y, _, _ = g.get_state()
    np.testing.assert_allclose(x, np.clip(np.zeros(inst.n), inst.l, inst.u), rtol=1e-15, atol=0)
    assert not np.any(y)
    g.close()


@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("k", [1, 100, 1000])
def test_fixed_step_iterates_match_oracle(name, k):
    compare_after(INSTANCES[name], k, replay=False, adaptive_step=False, restarts=False)


@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("k", [1, 10, 100, 1000])
def test_adaptive_iterates_match_oracle_on_device_decisions(name, k):
    compare_after(INSTANCES[name], k, tol=TOL if k <= 100 else TOL_LONG)


@pytest.mark.parametrize("name", ["open_300x600", "open_wide_3kx6k", "standard_form_500x1500"])
def test_wide_and_staged_forms_match_oracle(name):
    """The wide-tile forms (plain loads and staged) against the oracle after 300
    fixed-step FP64 attempts."""
    inst = INSTANCES[name]
    for form in (2, 3):
        g, o = pair(inst, prefetch=form, adaptive_step=False, restarts=False)
        g.pdhg_solve(0.0, 300)
        o.solve(0.0, 300)
        assert rel_err(g.primal(), o.primal()) <= TOL, (form, rel_err(g.primal(), o.primal()))
        assert rel_err(g.dual(), o.dual()) <= TOL, (form, rel_err(g.dual(), o.dual()))
        g.close()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("forms", [(1, 4), (2, 3)])
def test_kernel_forms_on_the_same_tiles_identical(precision, forms):
    inst = INSTANCES["open_300x600"]
    gs = [pair(inst, precision=precision, prefetch=f)[0] for f in forms]
    rs = [g.pdhg_solve(1e-6, 20000) for g in gs]
    assert rs[1].iterations == rs[0].iterations and rs[1].status == rs[0].status
    np.testing.assert_array_equal(gs[1].primal(), gs[0].primal())
    np.testing.assert_array_equal(gs[1].dual(), gs[0].dual())
    for g in gs:
        g.close()


@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("form", [0, 2])
def test_fp64_converges_to_the_constructed_optimum(name, form):
    inst = INSTANCES[name]
    g, _ = pair(inst, prefetch=form)
    r = g.pdhg_solve(1e-8, 400000)
    assert r.status == O.CONVERGED and r.rel_kkt <= 1e-8
    fs = inst.meta["f_star"]
    assert abs(r.pobj - fs) <= 1e-6 * (1 + abs(fs)) and abs(r.dobj - fs) <= 1e-6 * (1 + abs(fs))
    g.close()


@pytest.mark.parametrize("name", list(INSTANCES))
@pytest.mark.parametrize("form", [0, 2])
def test_mixed_precision_reaches_1e4_with_a_dual_residual(name, form):
    """FP32 bulk, FP64 checks: rel-KKT <= 1e-4 confirmed by the oracle's FP64
    evaluation of the returned point; objective within OBJ_TOL_MIXED of the
    constructed optimum; the solve passes through points whose dual residual is not
    zero (the one-sided and free columns' reduced costs)."""
    inst = INSTANCES[name]
    g, o = pair(inst, precision=1, prefetch=form)
    r0 = g.pdhg_solve(0.0, 64)
    assert r0.eps_d > 0.0
    g.reset_state()
    r = g.pdhg_solve(1e-4, 200000)
    assert r.status == O.CONVERGED and r.rel_kkt <= 1e-4
    x, y, _, _ = g.get_state()
    o.set_state(x, y)
    ev = o.evaluate(o.x, o.y)
    assert ev.rel_kkt <= 1.2e-4, ev
    assert abs(ev.eps_d - r.eps_d) <= 1e-6 + 1e-3 * ev.eps_d, (ev.eps_d, r.eps_d)
    fs = inst.meta["f_star"]
    assert abs(ev.pobj - fs) / (1 + abs(fs)) <= OBJ_TOL_MIXED
    g.close()


def test_persistent_kernel_converges_to_the_constructed_optimum():
    inst = INSTANCES["open_2kx4k"]
    g, _ = pair(inst, use_graph=3)
    r = g.pdhg_solve(1e-7, 200000)
    assert r.status == O.CONVERGED and r.launches == 2
    fs = inst.meta["f_star"]
    assert abs(r.pobj - fs) <= 1e-5 * (1 + abs(fs))
    g.close()


def test_batched_and_single_solves_agree_on_open_bounds():
    """The batched path (each LP its own step size, restarts and termination) on
    LPs with infinite column bounds: every LP matches its own single-LP solve after
    fixed-step attempts (1e-12) and converges to the constructed optimum."""
    S = lib()
    insts = [I.open_bounds_lp(200 + 150 * b, 400 + 300 * b, per_col=5, seed=40 + b) for b in range(5)]
    p = dict(adaptive_step=0, restarts=0)
    B = S.Batch(insts, S.default_params(precision=0, **p))
    B.solve(0.0, 200)
    for b, inst in enumerate(insts):
        g, o = pair(inst, adaptive_step=False, restarts=False)
        g.pdhg_solve(0.0, 200)
        o.solve(0.0, 200)
        assert rel_err(B.primal(b), g.primal()) <= 1e-12
        assert rel_err(B.primal(b), o.primal()) <= TOL
        g.close()
    B.close()
    B = S.Batch(insts, S.default_params(precision=0))
    res, _ = B.solve(1e-8, 400000)
    for r, inst in zip(res, insts):
        fs = inst.meta["f_star"]
        assert r.status == O.CONVERGED and abs(r.pobj - fs) <= 1e-6 * (1 + abs(fs))
    B.close()


@pytest.mark.parametrize("use_graph", [1, 3])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["open_bounds", "packcover", "mcf"])
def test_reported_errors_are_the_oracles_evaluation_of_the_returned_pair(name, precision, use_graph):
    """A solve reports the errors its last check measured (Section 2.2): they equal the
    oracle's FP64 evaluation of the pair the handle returns, within 1e-10 (1 + |value|),
    for eps_p, eps_d, eps_g and both objectives, in both precisions, for the chunk
    graphs and the persistent kernel, on LPs with and without free and one-sided
    columns (a nonzero dual residual on the first)."""
    inst = {"open_bounds": lambda: I.open_bounds_lp(300, 500, seed=4),
            "packcover": lambda: I.packing_covering(m=2000, n=4000, per_col=6, seed=9),
            "mcf": lambda: I.mcf(nodes=30, avg_degree=4, commodities=6, seed=2)}[name]()
    g, o = pair(inst, precision=precision, use_graph=use_graph)
    r = g.pdhg_solve(1e-6 if precision == 0 else 1e-4, 200000)
    assert r.status == O.CONVERGED
    ev = o.evaluate(g.primal() / o.C, g.dual() / o.R)
    for key, a, b in (("eps_p", r.eps_p, ev.eps_p), ("eps_d", r.eps_d, ev.eps_d), ("eps_g", r.eps_g, ev.eps_g),
                      ("pobj", r.pobj, ev.pobj), ("dobj", r.dobj, ev.dobj)):
        assert abs(a - b) <= 1e-10 * (1 + abs(b)), (key, a, b)
    if name == "open_bounds":
        assert ev.eps_d > 0.0
    g.close()
