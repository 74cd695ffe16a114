"""The multi-GPU path of bench.py on CPU: two ranks over the gloo backend.

Each rank solves its own seeded LP (weak scaling) and the only exchange is the
whole-job reduction of the timings (slowest rank) and of the work done (sum over
ranks).  These tests run that reduction and the per-rank workload choice in two
processes on 127.0.0.1; no GPU is touched.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, init_method=f"tcp://127.0.0.1:{port}")
    try:
        times = (1.0 + rank, 10.0 - rank, 0.5 * (rank + 1))
        counts = (448 + rank, 448, 7 + 2 * rank)
        t, c = bench.combine_ranks(dist, times, counts, "cpu")
        out[rank] = (t, c)
    finally:
        dist.destroy_process_group()


def test_whole_job_reduction_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork of this (threaded) test process
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        t, c = res[rank]
        assert t == [2.0, 10.0, 1.0]  # slowest rank per timed region
        assert c == [897.0, 896.0, 16.0]  # total work over the ranks


def test_single_process_reduction_is_identity():
    import bench
    t, c = bench.combine_ranks(None, (1.5, 2.5), (3, 4), "cpu")
    assert t == [1.5, 2.5] and c == [3.0, 4.0]


def test_each_rank_solves_its_own_seeded_lp_of_the_same_shape():
    import bench
    a, b = bench.instance(0), bench.instance(1)
    assert (a.m, a.n) == (b.m, b.n) == (50_000, 100_000)
    assert abs(a.nnz - b.nnz) <= 0.01 * a.nnz
    assert not (a.csr().indices[:1000] == b.csr().indices[:1000]).all()
