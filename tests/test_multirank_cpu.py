"""The bench's multi-process path on CPU ranks (gloo, world size 2): the path
runs as independent replicas, one tensor per rank with no collective on the
data path, so the only cross-rank steps are the max-over-ranks time and the
whole-job throughput built from it; every rank also builds the same seeded
workload."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], dist, torch.device("cpu"))
        A, _, _ = bench.make_inputs()
        digest = float(np.asarray(A, dtype=np.float64)[::97, ::13, ::17].sum())
        q.put((rank, t, bench.job_throughput(world, 3, t), digest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, times = 2, [12.5, 17.25]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [max(times)] * world
    # whole-job throughput: both ranks' entries over the slowest rank's time
    entries = bench.L * bench.M * bench.N * 3
    assert out[0][2] == pytest.approx(world * entries / (max(times) / 1e3), rel=1e-12)
    assert out[0][2] == out[1][2]
    assert out[0][3] == out[1][3]          # identical seeded replicas


def test_single_process_is_unchanged():
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.job_throughput(1, 2, 1000.0) == pytest.approx(2 * bench.L * bench.M * bench.N)
