"""K-objective fan-out (one LP, K pump objectives as SpMM PDHG) against per-objective
single-LP solves and the oracle.

Objective k of a fan-out is the Section 2.4 update around rounding target k.  In the
fixed-step mode its iterates after fixed attempt counts match the oracle's PDHG on
that objective within 1e-9 and the single-LP GPU solve within 1e-10 (the SpMM sums a
row with fused multiply-adds, the warp-tile SpMV with rounded products); in the
adaptive mode every objective converges on its own to the single solve's objective;
FP32-mixed fan-outs reach relative KKT 1e-4.
"""
import numpy as np
import pytest

from oracle import pdhg as O
from oracle import pump as P
from paper_2307_03466_gb300 import instances as I
from tests.gpu_common import gpu_available, lib, rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def setup(K=6, precision=0, **kw):
    S = lib()
    inst = I.packing_covering(m=400, n=900, per_col=6, int_frac=0.4, seed=31, binary=True, name="fan_small")
    params = S.default_params(precision=precision, aux_general_integers=0, **kw)
    base = S.LP.from_instance(inst, params)
    base.pdhg_solve(1e-3, 5000)  # the warm start every objective shares
    x = base.primal()
    target = x.copy()
    ic = inst.is_int == 1
    target[ic] = np.floor(x[ic] + 0.5)
    targets = I.fanout_targets(inst, target, K=K, flip_frac=0.1, seed=7)
    xs, ys, eta, om = base.get_state()
    return S, inst, base, targets, (xs, ys, eta, om), params


def single(S, inst, params, state, target, k, tol=0.0):
    g = S.LP.from_instance(inst, params)
    g.set_state(*state)
    g.set_objective(target, 1)
    r = g.pdhg_solve(tol, k)
    return g, r


@pytest.mark.parametrize("k", [10, 200])
def test_fixed_step_fanout_matches_single_solves_and_oracle(k):
    S, inst, base, targets, state, params = setup(adaptive_step=0, restarts=0)
    F = S.Fanout(base, targets, round_K=1)
    res, _ = F.solve(0.0, k)
    for q in range(targets.shape[1]):
        assert res[q].iterations == k and res[q].status == O.ITER_LIMIT
        xf = F.primal(q)
        g, r = single(S, inst, params, state, targets[:, q], k)
        assert rel_err(xf, g.primal()) <= 1e-10, (q, rel_err(xf, g.primal()))
        g.close()
        o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u,
                       params=O.PdhgParams(adaptive_step=False, restarts=False))
        chat, _, off = P.objective_update(inst.c, inst.is_int, inst.l, inst.u, targets[:, q], 1, [])
        o.set_objective_vector(chat, off)
        o.set_state(state[0], state[1])
        o.eta, o.omega = state[2], state[3]
        o.solve(0.0, k)
        assert rel_err(xf, o.primal()) <= 1e-9, (q, rel_err(xf, o.primal()))
    F.close()
    base.close()


def test_adaptive_fanout_converges_like_single_solves():
    S, inst, base, targets, state, params = setup()
    F = S.Fanout(base, targets, round_K=1)
    res, sec = F.solve(1e-6, 200000)
    assert sec > 0
    for q in range(targets.shape[1]):
        assert res[q].status == O.CONVERGED and res[q].rel_kkt <= 1e-6, (q, res[q].status, res[q].rel_kkt)
        g, r = single(S, inst, params, state, targets[:, q], 200000, tol=1e-6)
        assert r.status == O.CONVERGED
        assert abs(res[q].pobj - r.pobj) <= 1e-5 * (1 + abs(r.pobj)), (q, res[q].pobj, r.pobj)
        g.close()
    F.close()
    base.close()


def test_mixed_fanout_reaches_1e4():
    S, inst, base, targets, state, params = setup(precision=1)
    F = S.Fanout(base, targets, round_K=2)
    res, _ = F.solve(1e-4, 200000)
    for q in range(targets.shape[1]):
        assert res[q].status == O.CONVERGED and res[q].rel_kkt <= 1e-4, q
        # the oracle re-evaluates the returned primal with the objective of target q
        o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
        chat, _, off = P.objective_update(inst.c, inst.is_int, inst.l, inst.u, targets[:, q], 2, [])
        o.set_objective_vector(chat, off)
        ref = o.solve(1e-8, 400000)
        assert abs(res[q].pobj - ref.pobj) <= 1e-3 * (1 + abs(ref.pobj)), q  # oracle at 1e-4: <= 8e-5
    F.close()
    base.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_reported_errors_are_the_oracles_evaluation_of_the_returned_pair(precision):
    """Each objective's result reports the errors its last check measured (FP64 sums;
    in FP32-mixed, sums kept as FP32 pairs good to about 2^-44 of the terms): they
    equal the oracle's FP64 evaluation (Section 2.2) of the returned pair (x, y)
    under that objective within 1e-10 (1 + |value|).  A pair sum without the low
    part of the FP64 entries (2^-24 per term) misses eps_p by about 1e-8 and the
    dual objective by about 1e-3 here."""
    S, inst, base, targets, state, params = setup(K=6, precision=precision)
    F = S.Fanout(base, targets, round_K=1)
    res, _ = F.solve(1e-6 if precision == 0 else 1e-4, 200000)
    for q in range(targets.shape[1]):
        assert res[q].status == O.CONVERGED, q
        o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
        chat, _, off = P.objective_update(inst.c, inst.is_int, inst.l, inst.u, targets[:, q], 1, [])
        o.set_objective_vector(chat, off)
        x, y = F.primal(q), F.dual(q)
        assert x.shape == (inst.n,) and y.shape == (inst.m,)
        ev = o.evaluate(x / o.C, y / o.R)
        r = res[q]
        for name, a, b in (("eps_p", r.eps_p, ev.eps_p), ("eps_d", r.eps_d, ev.eps_d), ("eps_g", r.eps_g, ev.eps_g),
                           ("pobj", r.pobj, ev.pobj), ("dobj", r.dobj, ev.dobj)):
            assert abs(a - b) <= 1e-10 * (1 + abs(b)), (q, name, a, b)
    with pytest.raises(S.ScyllaError):
        F.dual(targets.shape[1])
    F.close()
    base.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_reported_errors_with_free_and_one_sided_columns(precision):
    """The same on an LP with free, one-sided and fixed columns and every row kind
    (no integer columns, so the objectives coincide): the dual residual, which is
    exactly 0 where both bounds of a column are finite, is nonzero here and agrees with
    the oracle's, as do the other errors and both objectives."""
    S = lib()
    inst = I.open_bounds_lp(300, 500, seed=4)
    params = S.default_params(precision=precision, aux_general_integers=0)
    base = S.LP.from_instance(inst, params)
    base.pdhg_solve(1e-3, 20000)
    targets = np.repeat(base.primal()[:, None], 3, axis=1)
    F = S.Fanout(base, targets, round_K=1)
    res, _ = F.solve(1e-6 if precision == 0 else 1e-4, 200000)
    seen_eps_d = False
    for q in range(targets.shape[1]):
        assert res[q].status == O.CONVERGED, q
        o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
        chat, _, off = P.objective_update(inst.c, inst.is_int, inst.l, inst.u, targets[:, q], 1, [])
        o.set_objective_vector(chat, off)
        ev = o.evaluate(F.primal(q) / o.C, F.dual(q) / o.R)
        r = res[q]
        seen_eps_d |= ev.eps_d > 0.0
        for name, a, b in (("eps_p", r.eps_p, ev.eps_p), ("eps_d", r.eps_d, ev.eps_d), ("eps_g", r.eps_g, ev.eps_g),
                           ("pobj", r.pobj, ev.pobj), ("dobj", r.dobj, ev.dobj)):
            assert abs(a - b) <= 1e-10 * (1 + abs(b)), (q, name, a, b)
    assert seen_eps_d
    F.close()
    base.close()


def test_fanout_needs_lp_without_aux_columns():
    S = lib()
    inst = I.packing_covering(m=60, n=120, per_col=3, seed=3)  # general integers -> auxiliary columns
    lp = S.LP.from_instance(inst)
    assert lp.n_aux > 0
    with pytest.raises(S.ScyllaError) as ei:
        S.Fanout(lp, np.zeros((inst.n, 2)))
    assert ei.value.code == S.ERR_UNSUPPORTED
    lp.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_tile_shapes_identical_in_fixed_step_and_tuner_reports(precision):
    """The autotuner's tile shapes of the two SpMMs (objectives per lane, slots per
    sweep) compute every entry of x', y' and A x' with the same sums in the same
    order.  Only the order in which the per-objective step-size sums are reduced
    depends on the shape (rows per warp), and the fixed-step mode takes no decision
    from them: there every forced shape gives identical iterates.  The tuner reports
    the shapes it chose and its timings."""
    S, inst, base, targets, state, params = setup(K=40, precision=precision, adaptive_step=0, restarts=0)
    F = S.Fanout(base, targets, round_K=1)
    sp, sd, ms = F.info()
    valid = (1, 2, 3, 4) if precision == 1 else (2, 4)
    assert sp in valid and sd in valid
    assert all(ms[s - 1] > 0 and ms[4 + s - 1] > 0 for s in valid)
    xs = {}
    for shapes in [(a, b) for a in valid for b in valid]:
        F.tune(*shapes)
        assert F.info()[:2] == shapes
        F.solve(0.0, 150)
        xs[shapes] = np.stack([F.primal(q) for q in range(targets.shape[1])])
    ref = xs[(valid[0], valid[0])]
    for shapes, v in xs.items():
        np.testing.assert_array_equal(v, ref, err_msg=str(shapes))
    with pytest.raises(S.ScyllaError):
        F.tune(5, 0)
    if precision == 0:
        with pytest.raises(S.ScyllaError):
            F.tune(1, 0)  # FP64 takes shapes 2 and 4
    F.close()
    base.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_tile_shapes_converge_alike_with_rejections_and_restarts(precision):
    """Adaptive solves in every shape (rejected attempts and restarts to the average
    on the way, so the pool copies run) converge per objective to the single-LP
    solve's objective."""
    S, inst, base, targets, state, params = setup(K=40, precision=precision)
    F = S.Fanout(base, targets, round_K=1)
    valid = (1, 2, 3, 4) if precision == 1 else (2, 4)
    tol = 1e-6 if precision == 0 else 1e-4
    ref = {}
    for q in range(0, targets.shape[1], 7):
        g, r = single(S, inst, params, state, targets[:, q], 200000, tol=1e-8)
        ref[q] = r.pobj
        g.close()
    rej = rst = 0
    for shapes in [(s, s) for s in valid]:
        F.tune(*shapes)
        res, _ = F.solve(tol, 200000)
        rej += sum(r.rejected for r in res)
        rst += sum(r.restarts for r in res)
        for q, pobj in ref.items():
            assert res[q].status == O.CONVERGED, (shapes, q)
            assert abs(res[q].pobj - pobj) <= 10 * tol * (1 + abs(pobj)), (shapes, q, res[q].pobj, pobj)
    assert rej > 0 and rst > 0
    F.close()
    base.close()


def test_second_solve_continues_from_the_first():
    """A solve that stops at an iteration limit leaves every objective's pair in the
    current pool (finished objectives carried, averages copied in): a second solve
    continues from there, as one longer solve does, up to the restart schedule's
    dependence on the attempt count (same objectives converged, same answers)."""
    S, inst, base, targets, state, params = setup(K=8, precision=0)
    F = S.Fanout(base, targets, round_K=1)
    r1, _ = F.solve(1e-7, 128)
    r2, _ = F.solve(1e-7, 200000)
    for q in range(targets.shape[1]):
        assert r2[q].status == O.CONVERGED, q
        g, r = single(S, inst, params, state, targets[:, q], 200000, tol=1e-7)
        assert abs(r2[q].pobj - r.pobj) <= 1e-5 * (1 + abs(r.pobj)), q
        g.close()
    F.close()
    base.close()


def test_a_ranks_share_of_the_objectives_solves_as_in_the_whole_fanout():
    """On several GPUs each rank solves its share of the K objectives as one
    fan-out from the same warm start (paper_2307_03466_gb300.shard): in the
    fixed-step mode, with the tile shapes forced alike, every objective of a share
    ends exactly where it does in the whole fan-out."""
    from paper_2307_03466_gb300 import shard
    S, inst, base, targets, state, params = setup(K=12, adaptive_step=0, restarts=0)
    # the whole fan-out starts, like every share, from the warm start set through
    # set_state (the unscaled state scaled again, as a rank receives it)
    b1 = S.LP.from_instance(inst, params)
    b1.set_state(*state)
    F = S.Fanout(b1, targets, round_K=1)
    F.tune(2, 2)
    F.solve(0.0, 150)
    full = [F.primal(q) for q in range(targets.shape[1])]
    F.close()
    b1.close()
    for share in shard.partition([1.0] * targets.shape[1], 3):
        b2 = S.LP.from_instance(inst, params)
        b2.set_state(*state)
        G = S.Fanout(b2, targets[:, share], round_K=1)
        G.tune(2, 2)
        G.solve(0.0, 150)
        for q, k in enumerate(share):
            np.testing.assert_array_equal(G.primal(q), full[k])
        G.close()
        b2.close()
    base.close()
