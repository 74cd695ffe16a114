"""Splitting the independent units of the batched and fan-out workloads over the
ranks of a multi-GPU job (paper_2307_03466_gb300/shard.py), on CPU: the partition's
properties, and the per-rank solve plus gather to rank 0 over two gloo ranks.  The
solve is stubbed with the oracle's PDHG on small LPs (this test only), so rank 0
must receive exactly what one process computes for every unit."""
import os
import socket

import numpy as np
import pytest

from paper_2307_03466_gb300 import instances as I
from paper_2307_03466_gb300 import shard

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_covers_every_unit_once_and_balances(world):
    rng = np.random.default_rng(world)
    w = list(rng.pareto(1.5, size=57) + 1.0)
    parts = shard.partition(w, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(w)))
    for p in parts:
        assert p == sorted(p)
    loads = [sum(w[i] for i in p) for p in parts]
    # greedy by decreasing weight: the spread is at most the largest weight
    assert max(loads) - min(loads) <= max(w) + 1e-9
    assert shard.partition(w, world) == parts  # deterministic


def test_partition_of_the_batched_workload_by_cost():
    sizes = I.power_law_sizes()
    w = [float(2 * 8 * 2 * m + 3 * m) for m in sizes]  # 8 nonzeros per column, n = 2 m
    parts = shard.partition(w, 4)
    loads = [sum(w[i] for i in p) for p in parts]
    assert max(loads) / min(loads) < 1.05


def _oracle_solve(insts):
    from oracle import pdhg as O  # test-only stub of the per-rank solve

    def solve(idx):
        out = []
        for i in idx:
            inst = insts[i]
            o = O.OracleLP(inst.csr(), inst.c, inst.lo, inst.hi, inst.l, inst.u)
            r = o.solve(1e-6, 20000)
            out.append({"i": i, "status": r.status, "pobj": r.pobj, "x": o.primal().tolist()})
        return out
    return solve


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        insts = [I.tiny_lp(100 + s, m=6, n=9, density=0.5) for s in range(7)]
        res = shard.solve_sharded(shard.batch_weights(insts), _oracle_solve(insts), dist)
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_sharded_solve_gathers_every_result_on_rank_zero():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[1] is None
    insts = [I.tiny_lp(100 + s, m=6, n=9, density=0.5) for s in range(7)]
    ref = shard.solve_sharded(shard.batch_weights(insts), _oracle_solve(insts), None)
    got = res[0]
    assert [r["i"] for r in got] == list(range(7))
    for a, b in zip(got, ref):
        assert a["status"] == b["status"] and a["pobj"] == b["pobj"] and a["x"] == b["x"]


def test_fanout_objectives_split_evenly():
    parts = shard.partition([1.0] * 64, 8)
    assert [len(p) for p in parts] == [8] * 8
