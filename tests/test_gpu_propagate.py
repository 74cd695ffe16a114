"""Bound propagation on the GPU (scylla_propagate) against the oracle.

- Any data: domains, ignored rows, round and conflict counts equal the oracle's
  round-based propagation bit for bit (same visit arithmetic, same merge), from the
  column bounds and from partial fixings, on handles with and without auxiliary
  columns (which the propagation leaves out).
- Integer data without ignored rows or conflicts: the domains equal the sequential
  (FIFO) propagation's, the first step of fix-and-propagate.
- At the bench size the generator's interior point survives the propagation of a
  fixing that contains it.
"""
import numpy as np
import pytest

from oracle import fixprop as F
from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import gpu_available, lib, long_row_instance
from tests.test_oracle_propagation_rounds import integer_instance
from tests.test_oracle_fixprop import csr

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def handle(inst, **kw):
    S = lib()
    return S.LP.from_instance(inst, S.default_params(**kw))


def oracle_rounds(inst, dl, du):
    return F.propagate_rounds(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, dl, du, inst.is_int)


def as_instance(dense, lo, hi, l, u, is_int):
    rp, ci, v = csr(dense)
    n = dense.shape[1]
    return I.Instance("prop", dense.shape[0], n, np.asarray(rp, np.int64), np.asarray(ci, np.int32),
                      np.asarray(v, float), np.zeros(n), lo, hi, l, u, np.asarray(is_int, np.uint8))


def compare(inst, g, dl0, du0):
    dl, du, ign, rounds, conflicts = g.propagate(dl0, du0)
    ol, ou, oign, orounds, oconf = oracle_rounds(inst, dl0, du0)
    assert np.array_equal(dl, ol) and np.array_equal(du, ou)
    assert np.array_equal(ign, oign) and rounds == orounds and conflicts == oconf
    return dl, du, ign, rounds, conflicts


@pytest.mark.parametrize("seed", range(12))
def test_integer_data_equals_rounds_and_fifo(seed):
    dense, x0, lo, hi, l, u = integer_instance(seed, m=40, n=50)
    inst = as_instance(dense.astype(float), lo, hi, l, u, np.ones(dense.shape[1]))
    g = handle(inst)
    dl, du, ign, rounds, conflicts = compare(inst, g, inst.l, inst.u)
    if not ign.any() and conflicts == 0:
        fl, fu, _ = F.propagate_only(inst.rowptr, inst.cols, inst.vals, inst.lo, inst.hi, inst.l, inst.u,
                                     inst.is_int)
        assert np.array_equal(dl, fl) and np.array_equal(du, fu)
    assert np.all(dl <= x0) and np.all(x0 <= du)
    g.close()


@pytest.mark.parametrize("name", ["setcover", "knapcover", "packcover", "long_rows", "mcf_small"])
def test_mixed_data_and_partial_fixings_equal_rounds(name):
    inst = {"setcover": lambda: I.set_cover(),
            "knapcover": lambda: I.knapsack_cover(300, seed=8),
            "packcover": lambda: I.packing_covering(m=400, n=800, per_col=4, seed=21),
            "long_rows": lambda: long_row_instance(),
            "mcf_small": lambda: I.mcf(nodes=20, avg_degree=4, commodities=6, seed=2)}[name]()
    for aux in (0, 1):
        g = handle(inst, aux_general_integers=aux)
        compare(inst, g, inst.l, inst.u)
        # fix a quarter of the integer columns at a rounded interior value
        rng = np.random.default_rng(3)
        ic = np.nonzero(inst.is_int)[0]
        fix = rng.choice(ic, size=max(1, len(ic) // 4), replace=False) if len(ic) else np.array([], int)
        dl0, du0 = inst.l.copy(), inst.u.copy()
        hi_fin = np.where(np.isfinite(inst.u[fix]), inst.u[fix], inst.l[fix] + 3)
        v = np.floor(rng.uniform(inst.l[fix], hi_fin + 1))
        v = np.minimum(np.maximum(v, inst.l[fix]), inst.u[fix])
        dl0[fix] = v
        du0[fix] = v
        compare(inst, g, dl0, du0)
        g.close()


def test_bench_size_interior_point_survives():
    inst = I.packing_covering(m=50_000, n=100_000, per_col=10, seed=1002)
    x0 = inst.meta["x0"]
    g = handle(inst, precision=1, aux_general_integers=0)
    ic = inst.is_int == 1
    dl0, du0 = inst.l.copy(), inst.u.copy()
    dl0[ic] = x0[ic]  # fix every integer column at x0's (integral) value
    du0[ic] = x0[ic]
    dl, du, ign, rounds, conflicts = g.propagate(dl0, du0)
    assert not ign.any() and conflicts == 0 and rounds >= 1
    assert np.all(dl <= x0 + 1e-9) and np.all(x0 <= du + 1e-9)
    assert np.all(dl >= dl0) and np.all(du <= du0)
    g.close()
