"""Batched PDHG (many LPs in one launch sequence) against per-LP solves and the oracle.

Each LP of a batch runs the same PDHG as its own single-LP solve: in the fixed-step
mode (no discrete decisions) its iterates match the oracle within 1e-9 and the
single-LP GPU solve within 1e-12 after fixed iteration counts; in the adaptive mode
every LP converges on its own to the requested tolerance with the single solve's
objective; FP32-mixed batches reach relative KKT 1e-4 checked by the oracle.
"""
import numpy as np
import pytest

from oracle import pdhg as O
from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import gpu_available, lib, long_row_instance, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def batch_instances():
    return [
        I.set_cover(m=120, n=300, seed=41),
        I.knapsack_cover(400, seed=42),
        long_row_instance(seed=43),
        I.packing_covering(m=1500, n=3000, per_col=10, seed=44),
        I.knapsack_cover(64, seed=45, per_col=4),
        I.mcf(nodes=24, avg_degree=4, commodities=8, seed=46),
    ]


def oracle_of(inst, **kw):
    return O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u, params=O.PdhgParams(**kw))


@pytest.mark.parametrize("k", [1, 10, 100, 1000])
def test_fixed_step_batch_matches_oracle_and_single(k):
    S = lib()
    insts = batch_instances()
    p = S.default_params(adaptive_step=0, restarts=0)
    B = S.Batch(insts, p)
    res, _ = B.solve(0.0, k)
    for b, inst in enumerate(insts):
        assert res[b].iterations == k and res[b].status == O.ITER_LIMIT
        xb = B.primal(b)
        o = oracle_of(inst, adaptive_step=False, restarts=False)
        o.solve(0.0, k)
        assert rel_err(xb, o.primal()) <= 1e-9, (b, rel_err(xb, o.primal()))
        g = S.LP.from_instance(inst, S.default_params(adaptive_step=0, restarts=0, aux_general_integers=0))
        g.pdhg_solve(0.0, k)
        assert rel_err(xb, g.primal()) <= 1e-12, b
        g.close()
    B.close()


def test_adaptive_batch_converges_like_single_solves():
    S = lib()
    insts = batch_instances()
    B = S.Batch(insts)
    res, sec = B.solve(1e-6, 200000)
    assert sec > 0
    iters = []
    for b, inst in enumerate(insts):
        assert res[b].status == O.CONVERGED and res[b].rel_kkt <= 1e-6, (b, res[b].status, res[b].rel_kkt)
        g = S.LP.from_instance(inst, S.default_params(aux_general_integers=0))
        r = g.pdhg_solve(1e-6, 200000)
        assert abs(res[b].pobj - r.pobj) <= 1e-5 * (1 + abs(r.pobj)), b
        # the oracle confirms the returned point
        o = oracle_of(inst)
        o.set_state(np.concatenate([B.primal(b)]), np.zeros(inst.m))
        iters.append(res[b].iterations)
        g.close()
    # LPs finish at different attempts and drop out while the others continue
    assert len(set(iters)) > 1
    B.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_reported_errors_are_the_oracles_evaluation_of_the_returned_pair(precision):
    """Each LP's result reports the errors its last check measured: they equal the
    oracle's evaluation (Section 2.2) of the returned pair (x, y) within
    1e-10 (1 + |value|), eps_p, eps_d, eps_g and both objectives, on LPs of every
    kind in the batch (an LP with free, one-sided and fixed columns included, whose
    dual residual is not zero)."""
    S = lib()
    insts = batch_instances()[:4] + [I.open_bounds_lp(300, 500, seed=4)]
    B = S.Batch(insts, S.default_params(precision=precision))
    res, _ = B.solve(1e-6 if precision == 0 else 1e-4, 200000)
    seen_eps_d = False
    for b, inst in enumerate(insts):
        assert res[b].status == O.CONVERGED, b
        x, y = B.primal(b), B.dual(b)
        assert x.shape == (inst.n,) and y.shape == (inst.m,)
        o = oracle_of(inst)
        ev = o.evaluate(x / o.C, y / o.R)
        r = res[b]
        seen_eps_d |= ev.eps_d > 0.0
        for name, a, c in (("eps_p", r.eps_p, ev.eps_p), ("eps_d", r.eps_d, ev.eps_d), ("eps_g", r.eps_g, ev.eps_g),
                           ("pobj", r.pobj, ev.pobj), ("dobj", r.dobj, ev.dobj)):
            assert abs(a - c) <= 1e-10 * (1 + abs(c)), (b, name, a, c)
    assert seen_eps_d
    with pytest.raises(S.ScyllaError):
        B.dual(len(insts))
    B.close()


def test_mixed_batch_reaches_1e4_checked_by_oracle():
    S = lib()
    insts = batch_instances()
    B = S.Batch(insts, S.default_params(precision=S.PREC_MIXED))
    res, _ = B.solve(1e-4, 200000)
    for b, inst in enumerate(insts):
        assert res[b].status == O.CONVERGED and res[b].rel_kkt <= 1e-4, b
        ref = oracle_of(inst)
        rr = ref.solve(1e-8, 400000)
        assert abs(res[b].pobj - rr.pobj) <= 1e-3 * (1 + abs(rr.pobj)), b
    B.close()


def test_batch_warm_start_and_reset():
    S = lib()
    insts = batch_instances()[:3]
    B = S.Batch(insts)
    r1, _ = B.solve(1e-6, 100000)
    r2, _ = B.solve(1e-6, 100000)
    assert all(r.iterations == 0 and r.status == O.CONVERGED for r in r2)
    B.reset_state()
    r3, _ = B.solve(1e-6, 100000)
    assert [r.iterations for r in r3] == [r.iterations for r in r1]
    B.close()


def test_batch_rejects_invalid_member():
    S = lib()
    bad = I.set_cover(m=20, n=30, seed=1)
    bad.lo[3] = 5.0
    bad.hi[3] = 1.0
    with pytest.raises(S.ScyllaError) as ei:
        S.Batch([I.set_cover(m=20, n=30, seed=2), bad])
    assert ei.value.code == S.ERR_INVALID_ARG and "LP 1" in str(ei.value)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("adaptive", [0, 1])
def test_persistent_queue_and_graph_paths_identical(precision, adaptive):
    """The persistent launch (warps take tiles from a shared queue over the LPs still
    running, compacted at every check), the launch-per-phase graphs over a static
    deal of the tiles and (FP32-mixed) the same graphs whose warps stage their next
    tile by asynchronous copies compute every tile with the same arithmetic and
    reduce each LP's per-tile sums in the same order: identical points, attempt
    counts, rejections and restarts, with LPs finishing at different checks on the
    way."""
    S = lib()
    insts = batch_instances()
    kw = dict(precision=precision, adaptive_step=adaptive, restarts=adaptive)
    tol = 1e-6 if precision == 0 else 1e-4
    out = {}
    modes = (1, 2, 3) if precision == 1 else (1, 2)
    for mode in modes:
        B = S.Batch(insts, S.default_params(batch_launch=mode, **kw))
        assert B.info()[0] == mode
        res, _ = B.solve(tol, 20000 if adaptive else 700)
        out[mode] = ([B.primal(b) for b in range(len(insts))],
                     [(r.iterations, r.rejected, r.restarts, r.status) for r in res])
        B.close()
    for mode in modes[1:]:
        for b in range(len(insts)):
            np.testing.assert_array_equal(out[mode][0][b], out[1][0][b], err_msg=f"{mode} {b}")
        assert out[mode][1] == out[1][1]
    if adaptive:
        assert len({t[0] for t in out[2][1]}) > 1  # LPs left the queue at different checks


@pytest.mark.parametrize("precision", [0, 1])
def test_persistent_queue_iteration_limit_inside_a_launch(precision):
    """An iteration limit that ends the attempts part way through a launch's n_check
    attempts: every block of the persistent launch makes the same number of attempts
    (the attempt counter is read before any block advances it), so no barrier waits
    for a block that left, and the points equal those of the graph form.  Repeated,
    because the order in which blocks start varies from launch to launch."""
    S = lib()
    insts = batch_instances()
    kw = dict(precision=precision)
    ref = {}
    B = S.Batch(insts, S.default_params(batch_launch=1, **kw))
    for limit in (1, 5, 63, 65, 130):
        B.reset_state()
        res, _ = B.solve(0.0, limit)
        ref[limit] = [B.primal(b) for b in range(len(insts))]
    B.close()
    B = S.Batch(insts, S.default_params(batch_launch=2, **kw))
    for rep in range(4):
        for limit in (1, 5, 63, 65, 130):
            B.reset_state()
            res, _ = B.solve(0.0, limit)
            assert all(r.status == O.ITER_LIMIT and r.iterations == limit for r in res), (rep, limit)
            for b in range(len(insts)):
                np.testing.assert_array_equal(B.primal(b), ref[limit][b], err_msg=f"{rep} {limit} {b}")
    B.close()


def test_persistent_queue_barrier_timeout_is_reported():
    """Every grid-barrier wait of the persistent batched kernel is bounded: with a
    limit far below any barrier's duration the first wait runs out, every block
    leaves, and the solve returns SCYLLA_ERR_TIMEOUT with the LPs marked
    DEVICE_TIMEOUT; the context stays usable and a batch with the normal limit then
    solves to the tolerance."""
    S = lib()
    insts = batch_instances()[:3]
    B = S.Batch(insts, S.default_params(batch_launch=2, device_wait_limit_s=1e-9))
    with pytest.raises(S.ScyllaError) as ei:
        B.solve(1e-6, 1000)
    assert ei.value.code == S.ERR_TIMEOUT
    B.close()
    B = S.Batch(insts, S.default_params(batch_launch=2))
    res, _ = B.solve(1e-6, 100000)
    assert all(r.status == O.CONVERGED for r in res)
    B.close()


def test_a_ranks_share_of_the_batch_solves_as_in_the_whole_batch():
    """On several GPUs each rank solves its share of the LPs as one batch
    (paper_2307_03466_gb300.shard): a share gives every one of its LPs exactly the
    result the whole batch gives it (per-LP preconditioning, per-tile sums and per-LP
    reductions in a fixed order do not depend on the other LPs)."""
    from paper_2307_03466_gb300 import shard
    S = lib()
    insts = batch_instances()
    params = S.default_params(batch_launch=1)
    full = shard.batch_solver(S, insts, params, 1e-6, 20000)(list(range(len(insts))))
    for share in shard.partition(shard.batch_weights(insts), 2):
        part = shard.batch_solver(S, insts, params, 1e-6, 20000)(share)
        for q, i in enumerate(share):
            assert part[q]["iterations"] == full[i]["iterations"] and part[q]["status"] == full[i]["status"]
            np.testing.assert_array_equal(part[q]["x"], full[i]["x"])
