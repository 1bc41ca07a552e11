"""Several GPUs are independent replicas (frames do not interact): each rank
tracks frames of its own and rank 0 reports the clusters of all ranks over the
slowest rank's time.  The host logic of that, on world-size-2 gloo ranks on
the CPU (no GPU, no data exchange beyond the two reductions)."""
from __future__ import annotations

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms, n = bench.reduce_job([12.5, 20.0][rank], [1000, 1500][rank], world)
        out.put((rank, ms, n, bench.replica_frame_ids(rank, 3)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_job():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, ms, n, _ in res:
        assert ms == 20.0 and n == 2500  # slowest rank, clusters of both
    assert set(res[0][3]).isdisjoint(res[1][3])  # each rank its own frames
    assert res[0][3] == [0, 1, 2] and res[1][3] == [3, 4, 5]


def test_single_process_needs_no_collective():
    import bench

    assert bench.reduce_job(7.0, 123, 1) == (7.0, 123)
    assert bench.replica_frame_ids(0, 8) == list(range(8))
