"""Parity at the benchmark sizes, in the launch configuration bench.py times.

The packing/covering workload (m = 50k, n = 100k, 1M nonzeros; the bench step) and
the MCF-shaped workload (n = 8.8M, m = 1.8M, 25.6M nonzeros; the DRAM-resident
case, whose per-attempt kernels take the wide-tile form) are both small enough for
the oracle to run a few attempts:

- FP64: fixed-step attempts from the cold start against the oracle, every entry
  (1e-9), and on the packing/covering workload 32 adaptive attempts replayed on
  the device's decisions (the same check as the small parity instances).
- FP32-mixed (the bench configuration): one attempt from a seeded state inside the
  bounds against the oracle's FP64 attempt from the same state, every entry on the
  packing/covering workload and sampled columns and rows (computed one by one by
  the oracle) on the MCF workload, within FP32 rounding.
- FP32-mixed solves to rel-KKT 1e-4, the bench's stopping rule, re-evaluated by the
  oracle on the returned point.
- The batched workload (256 power-law LPs, 17.2M nonzeros) and the fan-out workload
  (m = 200k, n = 500k, 5M nonzeros, K = 64): fixed-step FP64 attempts of sampled LPs
  and objectives against the oracle within 1e-9, and the FP32-mixed bench
  configuration converging for every LP and objective, with the oracle's primal
  residual of sampled points.
"""
import numpy as np
import pytest

from oracle import pdhg as O
from oracle import pump as P
from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import gpu_available, pair, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

MIXED_TOL = 2e-5  # FP32 iterates and products, FP32 row sums of ~10-20 terms, one attempt


@pytest.fixture(scope="module")
def packcover():
    # the bench step's workload (bench.instance(0))
    return I.packing_covering(m=50_000, n=100_000, per_col=10, seed=1002)


@pytest.fixture(scope="module")
def mcf():
    return I.mcf()


def seeded_state(inst, seed):
    """A state inside the column bounds, and a small dual, from a seeded generator."""
    rng = np.random.default_rng(seed)
    x = np.clip(rng.uniform(-0.5, 1.5, inst.n) * np.where(np.isfinite(inst.u), np.maximum(inst.u, 1.0), 1.0),
                inst.l, inst.u)
    y = rng.normal(0.0, 0.1, inst.m)
    return x, y


def one_attempt(inst, precision, x0, y0, prefetch=0):
    """Device: one fixed-step attempt from (x0, y0); oracle: the same attempt in FP64
    (both take the oracle's own initial step size and primal weight)."""
    g, o = pair(inst, precision=precision, adaptive_step=False, restarts=False, prefetch=prefetch)
    eta, om = o.eta, o.omega
    g.set_state(x0, y0, eta, om)
    r = g.pdhg_solve(0.0, 1)
    assert r.iterations == 1
    x1, y1, _, _ = g.get_state()
    g.close()
    o.set_state(x0, y0)
    return x1, y1, o, eta, om


def test_packcover_fp64_fixed_step_from_cold_start(packcover):
    g, o = pair(packcover, adaptive_step=False, restarts=False)
    g.pdhg_solve(0.0, 32)
    o.solve(0.0, 32)
    xg, yg, _, _ = g.get_state()
    assert rel_err(xg, o.primal()) <= 1e-9 and rel_err(yg, o.dual()) <= 1e-9
    g.close()


def test_packcover_fp64_adaptive_on_device_decisions(packcover):
    """32 adaptive attempts (a check at the start and at the limit) replayed on the
    device's step-size and restart decisions.  The two sides sum rows in different
    orders; over longer runs at this size the rounding difference grows past 1e-9
    (4e-8 after 100 attempts), as it does past 100 attempts on the small instances."""
    from tests.test_gpu_pdhg import compare_after
    compare_after(packcover, 32)


def test_packcover_mixed_one_attempt_every_entry(packcover):
    x0, y0 = seeded_state(packcover, 7)
    x1, y1, o, eta, om = one_attempt(packcover, 1, x0, y0)
    xs, ys = o.pdhg_step(o.x, o.y, eta, om)
    assert rel_err(x1, o.primal(xs)) <= MIXED_TOL
    assert rel_err(y1, o.dual(ys)) <= MIXED_TOL


def test_packcover_mixed_solve_reaches_1e4_checked_by_oracle(packcover):
    g, o = pair(packcover, precision=1)
    r = g.pdhg_solve(1e-4, 100000)
    assert r.status == O.CONVERGED and r.rel_kkt <= 1e-4
    x, y, _, _ = g.get_state()
    ev = o.evaluate(x / o.C, y / o.R)
    assert ev.rel_kkt <= 1.2e-4, ev
    g.close()


def test_mcf_fp64_fixed_step_from_cold_start_wide_tiles(mcf):
    g, o = pair(mcf, adaptive_step=False, restarts=False)
    g.pdhg_solve(0.0, 4)
    o.solve(0.0, 4)
    xg, yg, _, _ = g.get_state()
    assert rel_err(xg, o.primal()) <= 1e-9 and rel_err(yg, o.dual()) <= 1e-9
    g.close()


@pytest.mark.parametrize("prefetch", [0, 3])
def test_mcf_mixed_one_attempt_sampled(mcf, prefetch):
    """prefetch 0: the automatic form (wide tiles, plain loads); 3: wide tiles staged
    in shared memory by bulk copies."""
    x0, y0 = seeded_state(mcf, 11)
    x1, y1, o, eta, om = one_attempt(mcf, 1, x0, y0, prefetch=prefetch)
    rng = np.random.default_rng(5)
    cols = np.sort(rng.choice(mcf.n, 4000, replace=False))
    rows = np.sort(rng.choice(mcf.m, 4000, replace=False))
    xs_c = o.primal_step_at(cols, o.x, o.y, eta, om)
    assert rel_err(x1[cols], xs_c * o.C[cols]) <= MIXED_TOL
    # the dual step of a row needs the oracle's whole new primal iterate
    xs_all, ys_all = o.pdhg_step(o.x, o.y, eta, om)
    ys_r = o.dual_step_at(rows, o.x, xs_all, o.y, eta, om)
    np.testing.assert_allclose(ys_r, ys_all[rows], rtol=1e-13, atol=0)
    assert rel_err(y1[rows], ys_r * o.R[rows]) <= MIXED_TOL
    # and every entry, against the oracle's whole attempt
    assert rel_err(x1, o.primal(xs_all)) <= MIXED_TOL and rel_err(y1, o.dual(ys_all)) <= MIXED_TOL


def test_packcover_repair_of_a_feasible_fixing(packcover):
    """Continuous repair at the bench size: the integers fixed at those of the
    generator's interior point x0 (so the fixed LP is feasible and x0 is one of its
    points), solves to rel-KKT 1e-7 with the shift rounds (one solve leaves single
    rows outside the check's tolerance at this size).  The repaired point passes the
    oracle's exact feasibility test, keeps the fixed integers, and its objective is
    no worse than x0's."""
    from oracle import pump as P
    g, _ = pair(packcover, precision=1)
    x0 = packcover.meta["x0"]
    r, x = g.repair(x0, 1e-7, 100000)
    assert r.status == P.FOUND and r.rel_kkt <= 1e-7
    isi = packcover.is_int == 1
    assert np.array_equal(x[isi], x0[isi])
    assert P.check_feasible(packcover.rowptr, packcover.cols, packcover.vals, packcover.lo, packcover.hi,
                            packcover.l, packcover.u, packcover.is_int, x)
    assert float(packcover.c @ x) <= float(packcover.c @ x0) + 1e-6 * abs(float(packcover.c @ x0))
    g.close()


# ---- the batched and fan-out workloads of bench.py, at their full sizes ----------

def sampled(insts):
    """The smallest, a middle and the largest LP of a batch."""
    order = sorted(range(len(insts)), key=lambda b: insts[b].nnz)
    return [order[0], order[len(order) // 2], order[-1]]


def test_batch_bench_size_fixed_step_sampled_lps_match_oracle():
    """The 256 power-law LPs (17.2M nonzeros) as one batch: 8 fixed-step FP64 attempts;
    the smallest, a middle and the largest LP equal the oracle's PDHG within 1e-9."""
    from paper_2307_03466_gb300 import scylla as S
    insts = I.batch()
    assert len(insts) == 256
    B = S.Batch(insts, S.default_params(adaptive_step=0, restarts=0))
    res, _ = B.solve(0.0, 8)
    assert all(r.iterations == 8 for r in res)
    for b in sampled(insts):
        inst = insts[b]
        o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u,
                       params=O.PdhgParams(adaptive_step=False, restarts=False))
        o.solve(0.0, 8)
        assert rel_err(B.primal(b), o.primal()) <= 1e-9, b
    B.close()


def test_batch_bench_size_mixed_all_converge_primal_checked_by_oracle():
    """The bench configuration (FP32-mixed, rel-KKT 1e-4): every LP converges, and the
    oracle's primal residual of the sampled LPs' points agrees."""
    from paper_2307_03466_gb300 import scylla as S
    insts = I.batch()
    B = S.Batch(insts, S.default_params(precision=S.PREC_MIXED))
    res, _ = B.solve(1e-4, 200000)
    assert all(r.status == O.CONVERGED and r.rel_kkt <= 1e-4 for r in res)
    for b in sampled(insts):
        inst = insts[b]
        o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
        ev = o.evaluate(B.primal(b) / o.C, np.zeros(inst.m))
        assert ev.eps_p <= 1.2e-4, (b, ev.eps_p)
    B.close()


@pytest.fixture(scope="module")
def fan():
    """The fan-out workload of bench.py: m = 200k, n = 500k, 5M nonzeros, K = 64 targets
    around the rounded warm start (FP64 fixed-step base for the parity case)."""
    from paper_2307_03466_gb300 import scylla as S
    inst = I.fanout_base()
    return S, inst


def fan_targets(S, inst, base):
    base.pdhg_solve(1e-3, 20000)
    x = base.primal()
    target = x.copy()
    ic = inst.is_int == 1
    target[ic] = np.floor(x[ic] + 0.5)
    return I.fanout_targets(inst, target, K=64, flip_frac=0.10), base.get_state()


def test_fanout_bench_size_fixed_step_sampled_objectives_match_oracle(fan):
    S, inst = fan
    base = S.LP.from_instance(inst, S.default_params(aux_general_integers=0, adaptive_step=0, restarts=0))
    targets, state = fan_targets(S, inst, base)
    F = S.Fanout(base, targets, round_K=1)
    res, _ = F.solve(0.0, 4)
    assert all(r.iterations == 4 for r in res)
    o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u,
                   params=O.PdhgParams(adaptive_step=False, restarts=False))
    for q in (0, 31, 63):
        chat, _, off = P.objective_update(inst.c, inst.is_int, inst.l, inst.u, targets[:, q], 1, [])
        o.set_objective_vector(chat, off)
        o.set_state(state[0], state[1])
        o.eta, o.omega = state[2], state[3]
        o.solve(0.0, 4)
        assert rel_err(F.primal(q), o.primal()) <= 1e-9, q
    F.close()
    base.close()


def test_fanout_bench_size_mixed_all_converge_checked_by_oracle(fan):
    S, inst = fan
    base = S.LP.from_instance(inst, S.default_params(precision=S.PREC_MIXED, aux_general_integers=0))
    targets, _ = fan_targets(S, inst, base)
    F = S.Fanout(base, targets, round_K=1)
    res, _ = F.solve(1e-4, 200000)
    assert all(r.status == O.CONVERGED and r.rel_kkt <= 1e-4 for r in res)
    for q in (0, 63):
        o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
        chat, _, off = P.objective_update(inst.c, inst.is_int, inst.l, inst.u, targets[:, q], 1, [])
        o.set_objective_vector(chat, off)
        ev = o.evaluate(F.primal(q) / o.C, F.dual(q) / o.R)
        assert ev.rel_kkt <= 1.2e-4, (q, ev)
        for a, b in ((res[q].eps_p, ev.eps_p), (res[q].eps_d, ev.eps_d), (res[q].eps_g, ev.eps_g)):
            assert abs(a - b) <= 1e-10 * (1 + b), (q, a, b)
    F.close()
    base.close()


@pytest.fixture(scope="module")
def open_bounds_1m():
    # the packing/covering workload's size (m = 50k, n = 100k, 1M nonzeros) with
    # lower-only, upper-only, free and fixed columns and every row kind
    return I.open_bounds_lp(50_000, 100_000, per_col=10, seed=1012)


@pytest.mark.parametrize("prefetch", [0, 2])
def test_open_bounds_1m_fp64_fixed_step_both_forms(open_bounds_1m, prefetch):
    """100 fixed-step FP64 attempts from the cold start (checks at 64 and 100, so the
    column check's one-sided and free branches run) against the oracle, every entry
    within 1e-9: the automatic form (32-row tiles at this size, as in the bench) and
    the wide-tile form."""
    inst = open_bounds_1m
    g, o = pair(inst, adaptive_step=False, restarts=False, prefetch=prefetch)
    rg = g.pdhg_solve(0.0, 100)
    ro = o.solve(0.0, 100)
    xg, yg, _, _ = g.get_state()
    assert rel_err(xg, o.primal()) <= 1e-9 and rel_err(yg, o.dual()) <= 1e-9
    assert abs(rg.eps_d - ro.eps_d) <= 1e-9 * max(1.0, ro.eps_d) and ro.eps_d > 0
    assert abs(rg.eps_p - ro.eps_p) <= 1e-9 * max(1.0, ro.eps_p)
    assert abs(rg.eps_g - ro.eps_g) <= 1e-9 * max(1.0, ro.eps_g)
    g.close()


def test_open_bounds_1m_mixed_solve_reaches_1e4(open_bounds_1m):
    """The bench configuration (FP32-mixed, automatic form) on the same LP: rel-KKT
    <= 1e-4 confirmed by the oracle's FP64 evaluation, objective within 1e-3 of the
    constructed optimum."""
    inst = open_bounds_1m
    g, o = pair(inst, precision=1)
    r = g.pdhg_solve(1e-4, 200000)
    assert r.status == O.CONVERGED and r.rel_kkt <= 1e-4
    x, y, _, _ = g.get_state()
    ev = o.evaluate(x / o.C, y / o.R)
    assert ev.rel_kkt <= 1.2e-4, ev
    fs = inst.meta["f_star"]
    assert abs(ev.pobj - fs) / (1 + abs(fs)) <= 1e-3
    g.close()
