"""Infeasibility detection on the device against the oracle's detector and the
independent tests of a certificate.

The device tests the change of y since an anchor check as a candidate dual ray at
every check and ends the solve INFEASIBLE when D > 1e-9 S (D and S as in
oracle/infeas.py).  Checked here:
* built infeasible LPs (a feasible LP plus a row that only a combination of rows
  contradicts) end INFEASIBLE, with a ray that the oracle's test and the library's
  host test both confirm (D > 0), in FP64 and FP32-mixed, and at a size of many
  tiles; with a fixed step size at the same attempt and with the same ray as the
  oracle's detector on the device's decisions;
* the device's D and S of its last candidate equal the oracle's values of the same
  ray, on feasible LPs with free rows and columns (infinite terms included);
* on feasible LPs the detector never fires and changes nothing (bit-identical
  points in every launch mode);
* the API's errors (a handle without the detector, a batch asking for it).
"""
import math

import numpy as np
import pytest

from oracle import infeas as X
from oracle import pdhg as O
from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import gpu_available, lib
from tests.test_oracle_infeas import _built_infeasible

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

INF = np.inf


def _csr_parts(A):
    A = A.tocsr()
    return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)


def device_lp(A, c, lo, hi, l, u, precision=0, **kw):
    S = lib()
    p = S.default_params(precision=precision, aux_general_integers=0, infeasibility_checks=1, **kw)
    rp, ci, va = _csr_parts(A)
    m, n = A.shape
    return S.LP(rp, ci, va, c, lo, hi, l, u, np.zeros(n, np.uint8), m, n, p)


def _certificate_checks(g, A2, lo2, hi2, inst):
    """The device's ray passes the oracle's test and the library's compensated host
    test, and the device's D and S equal the oracle's D and S of that ray."""
    y, gap, scale = g.certificate()
    g_or, s_or = X.farkas_gap_scale(A2, lo2, hi2, inst.l, inst.u, y)
    assert g_or > 0 and g.farkas_gap(y) > 0
    assert abs(gap - g_or) <= 1e-9 * s_or and abs(scale - s_or) <= 1e-9 * s_or
    assert gap > 1e-9 * scale
    return y


@pytest.mark.parametrize("seed", range(6))
def test_fixed_step_detection_at_the_oracles_check(seed):
    """FP64, fixed step size (the iteration is non-expansive, so the device's and the
    oracle's iterates stay within rounding of each other): the device ends
    INFEASIBLE after the same number of attempts as the oracle's detector on the
    device's step and restart decisions, with the same ray (1e-6)."""
    S = lib()
    inst, A2, lo2, hi2 = _built_infeasible(seed, *((40, 80) if seed < 4 else (120, 240)))
    g = device_lp(A2, inst.c, lo2, hi2, inst.l, inst.u, adaptive_step=0, trace_capacity=20000)
    r = g.pdhg_solve(1e-8, 20000)
    assert r.status == S.INFEASIBLE
    y = _certificate_checks(g, A2, lo2, hi2, inst)
    steps, checks = g.trace()
    o = O.OracleLP(A2, inst.c, lo2, hi2, inst.l, inst.u,
                   params=O.PdhgParams(infeasibility_checks=True, adaptive_step=False))
    ro = o.solve(1e-8, 20000, trace=True, replay=(steps, checks))
    assert ro.status == O.INFEASIBLE and ro.iterations == r.iterations
    assert np.max(np.abs(y - ro.certificate)) <= 1e-6 * np.max(np.abs(ro.certificate))
    g.close()


@pytest.mark.parametrize("seed", range(6))
def test_adaptive_detection_gives_a_certificate(seed):
    """FP64, adaptive step size: the device ends INFEASIBLE with a ray that both
    tests confirm, and the oracle's own adaptive solve ends INFEASIBLE too.  The
    attempt counts are not compared: with adaptive steps the iterates of an
    infeasible LP depend on rounding (in the oracle alone, a 1e-14 perturbation of
    the start point changes the candidate rays at O(1) within five checks, on the
    same decisions)."""
    S = lib()
    inst, A2, lo2, hi2 = _built_infeasible(seed, *((40, 80) if seed < 4 else (120, 240)))
    g = device_lp(A2, inst.c, lo2, hi2, inst.l, inst.u)
    r = g.pdhg_solve(1e-8, 5000)
    assert r.status == S.INFEASIBLE
    _certificate_checks(g, A2, lo2, hi2, inst)
    o = O.OracleLP(A2, inst.c, lo2, hi2, inst.l, inst.u, params=O.PdhgParams(infeasibility_checks=True))
    assert o.solve(1e-8, 5000).status == O.INFEASIBLE
    g.close()


@pytest.mark.parametrize("seed", range(3))
def test_built_infeasible_lp_detected_in_mixed_precision(seed):
    """FP32-mixed: the detector works on the FP32 iterates (differences and sums in
    FP64) and its ray passes both tests."""
    S = lib()
    inst, A2, lo2, hi2 = _built_infeasible(seed, 120, 240)
    g = device_lp(A2, inst.c, lo2, hi2, inst.l, inst.u, precision=1)
    r = g.pdhg_solve(1e-8, 20000)
    assert r.status == S.INFEASIBLE
    y, gap, scale = g.certificate()
    assert X.farkas_gap(A2, lo2, hi2, inst.l, inst.u, y) > 0 and g.farkas_gap(y) > 0
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_built_infeasible_lp_of_many_tiles(precision):
    """A packing/covering LP of 6000 rows and 12000 columns plus the contradicting row
    (many blocks in both detector kernels, ragged last blocks)."""
    S = lib()
    inst = I.packing_covering(m=6000, n=12000, per_col=6, seed=321)
    rng = np.random.default_rng(5)
    A = inst.csr()
    ys = np.where(np.isfinite(inst.lo) & (rng.random(inst.m) < 0.5), rng.random(inst.m), 0.0)
    ys = np.where(np.isfinite(inst.hi) & (ys == 0.0), -rng.random(inst.m), ys)
    ys = np.where(((ys > 0) & ~np.isfinite(inst.lo)) | ((ys < 0) & ~np.isfinite(inst.hi)), 0.0, ys)
    L = X._side_min(ys, inst.lo, inst.hi)
    assert math.isfinite(L)
    import scipy.sparse as sp
    A2 = sp.vstack([A, sp.csr_matrix(A.T @ ys)]).tocsr()
    lo2, hi2 = np.append(inst.lo, -INF), np.append(inst.hi, L - 1.0)
    assert X.farkas_gap(A2, lo2, hi2, inst.l, inst.u, np.append(ys, -1.0)) > 0
    g = device_lp(A2, inst.c, lo2, hi2, inst.l, inst.u, precision=precision)
    r = g.pdhg_solve(1e-8, 40000)
    assert r.status == S.INFEASIBLE
    y, gap, scale = g.certificate()
    g_or, s_or = X.farkas_gap_scale(A2, lo2, hi2, inst.l, inst.u, y)
    assert g_or > 0 and g.farkas_gap(y) > 0
    assert abs(gap - g_or) <= 1e-9 * s_or
    g.close()


def test_row_against_its_box():
    S = lib()
    import scipy.sparse as sp
    A = sp.csr_matrix(np.array([[1.0, 1.0], [1.0, -1.0]]))
    lo, hi = np.array([3.0, -1.0]), np.array([INF, 1.0])
    g = device_lp(A, np.array([1.0, 2.0]), lo, hi, np.zeros(2), np.ones(2))
    r = g.pdhg_solve(1e-8, 5000)
    assert r.status == S.INFEASIBLE
    y, _, _ = g.certificate()
    assert X.farkas_gap(A, lo, hi, np.zeros(2), np.ones(2), y) > 0
    g.close()


@pytest.mark.parametrize("name", ["open_bounds", "packcover", "mcf"])
@pytest.mark.parametrize("precision", [0, 1])
def test_device_gap_and_scale_equal_the_oracles_for_the_same_ray(name, precision):
    """After 192 attempts of a feasible LP the last candidate (y at 192 minus y at 128)
    was tested: the device's D and S equal the oracle's D and S of that ray within
    1e-9 S (-inf on both sides when a term needs an infinite bound), and D <= 0."""
    inst = {"open_bounds": lambda: I.open_bounds_lp(300, 500, seed=4),
            "packcover": lambda: I.packing_covering(m=2000, n=4000, per_col=6, seed=9),
            "mcf": lambda: I.mcf(nodes=30, avg_degree=4, commodities=6, seed=2)}[name]()
    g = device_lp(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u, precision=precision)
    g.pdhg_solve(0.0, 192)
    y, gap, scale = g.certificate()
    assert np.any(y != 0.0)
    g_or, s_or = X.farkas_gap_scale(inst.csr(), inst.lo, inst.hi, inst.l, inst.u, y)
    if g_or == -math.inf:
        assert gap == -math.inf
    else:
        assert abs(gap - g_or) <= 1e-9 * s_or and abs(scale - s_or) <= 1e-9 * s_or
        assert gap <= 1e-9 * scale
    g.close()


@pytest.mark.parametrize("use_graph", [0, 1, 2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_detector_changes_nothing_on_feasible_lps(use_graph, precision):
    """With the detector on, feasible LPs solve bit for bit as without it (status,
    attempts, points), whatever the launch mode; the persistent mode (use_graph = 3)
    runs as chunk graphs then, so it is compared with the chunk graphs without it."""
    S = lib()
    for inst in (I.set_cover(m=120, n=300, seed=41), I.open_bounds_lp(200, 400, seed=7),
                 I.mcf(nodes=16, avg_degree=4, commodities=4, seed=3)):
        out = []
        for on in (0, 1):
            mode = 1 if (use_graph == 3 and not on) else use_graph
            p = S.default_params(precision=precision, aux_general_integers=0, infeasibility_checks=on,
                                 use_graph=mode)
            g = S.LP.from_instance(inst, p)
            r = g.pdhg_solve(1e-7 if precision == 0 else 1e-4, 4000)
            out.append((r.status, r.iterations, g.primal(), g.dual()))
            g.close()
        assert out[1][0] != S.INFEASIBLE
        assert out[0][:2] == out[1][:2]
        np.testing.assert_array_equal(out[0][2], out[1][2])
        np.testing.assert_array_equal(out[0][3], out[1][3])


def test_certificate_errors():
    S = lib()
    inst = I.set_cover(m=40, n=90, seed=2)
    g = S.LP.from_instance(inst, S.default_params(aux_general_integers=0))
    with pytest.raises(S.ScyllaError) as ei:
        g.certificate()
    assert ei.value.code == S.ERR_INVALID_ARG
    g.close()
    with pytest.raises(S.ScyllaError) as ei:
        S.Batch([inst, inst], S.default_params(infeasibility_checks=1))
    assert ei.value.code == S.ERR_UNSUPPORTED
    g = S.LP.from_instance(inst, S.default_params(aux_general_integers=0, infeasibility_checks=1))
    y, gap, scale = g.certificate()  # before any solve: nothing tested
    assert gap == -math.inf and scale == 0.0 and not np.any(y)
    g.close()
