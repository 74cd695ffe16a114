"""Independent units of work split over the ranks of a multi-GPU job.

Two workloads of the hot path are sets of independent problems with no exchange
between them while they are solved: the batched LP relaxations (each LP runs its
own PDHG, Sections 2.1-2.2 per LP) and the K pump objectives of a fan-out (each
objective its own PDHG on the same matrix, Section 2.4).  On several GPUs each
rank takes a share of the units, solves it on its own device with the
single-device path, and rank 0 collects the results; the only communication is
that final gather (and the timing reductions of a benchmark).

The partition is deterministic and depends only on the unit weights and the
number of ranks: units are dealt in order of decreasing weight, each to the rank
with the least total weight so far (ties to the lower rank), and every rank
keeps its units in ascending index order.  Weights are the units' costs per
attempt (nonzeros of an LP; equal for the objectives of a fan-out).

The solve itself is a callable passed in, ``solve(indices) -> list`` of per-unit
results in the order of ``indices``, so that this module holds no solver and the
partition and gather can be exercised on their own.
"""
from __future__ import annotations

from typing import Callable, Sequence


def partition(weights: Sequence[float], world: int) -> list:
    """Indices of the units of each rank (a list of ``world`` ascending lists)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-float(weights[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(weights[i])
    return [sorted(p) for p in parts]


def solve_sharded(weights: Sequence[float], solve: Callable[[list], list], dist=None) -> list | None:
    """Solve this rank's share and gather every unit's result on rank 0.

    dist: ``torch.distributed`` with an initialised process group, or None for one
    process.  Returns, on rank 0, the results of all units in index order; None on
    the other ranks.
    """
    if dist is None:
        idx = list(range(len(weights)))
        return list(solve(idx))
    world, rank = dist.get_world_size(), dist.get_rank()
    mine = partition(weights, world)[rank]
    res = list(solve(mine)) if mine else []
    if len(res) != len(mine):
        raise RuntimeError(f"rank {rank}: solve returned {len(res)} results for {len(mine)} units")
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(list(zip(mine, res)), gathered, dst=0)
    if rank != 0:
        return None
    out = [None] * len(weights)
    for part in gathered:
        for i, r in part:
            out[i] = r
    missing = [i for i, r in enumerate(out) if r is None]
    if missing:
        raise RuntimeError(f"units without a result after the gather: {missing[:8]}")
    return out


def batch_weights(instances) -> list:
    """Cost per attempt of each LP of a batch: its nonzeros (both sparse products
    read them once) plus its rows and columns (the vector passes)."""
    return [float(2 * inst.nnz + inst.m + inst.n) for inst in instances]


def batch_solver(S, instances, params, tol: float, iter_limit: int):
    """A ``solve(indices)`` for solve_sharded over the LPs of a batch: the LPs of the
    share as one batch on this rank's device (the library module S), each result a
    dict with status, attempts, objective, relative KKT error and the primal point."""
    def solve(idx):
        if not idx:
            return []
        B = S.Batch([instances[i] for i in idx], params)
        try:
            res, sec = B.solve(tol, iter_limit)
            return [{"status": int(r.status), "iterations": int(r.iterations), "pobj": float(r.pobj),
                     "rel_kkt": float(r.rel_kkt), "seconds": float(sec), "x": B.primal(q)}
                    for q, r in enumerate(res)]
        finally:
            B.close()
    return solve


def fanout_solver(S, instance, state, targets, round_K: int, params, tol: float, iter_limit: int):
    """A ``solve(indices)`` for solve_sharded over the K objectives of a fan-out: this
    rank builds the base LP from ``instance``, sets the shared warm start ``state``
    (x, y, eta, omega) and solves the objectives of its share (columns of
    ``targets``, n x K) as one fan-out."""
    def solve(idx):
        if not idx:
            return []
        base = S.LP.from_instance(instance, params)
        try:
            base.set_state(*state)
            F = S.Fanout(base, targets[:, idx], round_K=round_K)
            try:
                res, sec = F.solve(tol, iter_limit)
                return [{"status": int(r.status), "iterations": int(r.iterations), "pobj": float(r.pobj),
                         "rel_kkt": float(r.rel_kkt), "seconds": float(sec), "x": F.primal(q)}
                        for q, r in enumerate(res)]
            finally:
                F.close()
        finally:
            base.close()
    return solve
