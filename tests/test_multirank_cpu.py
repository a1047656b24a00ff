"""The multi-GPU path of bench.py on CPU ranks (gloo, world size 2): replicas with no data-path
collective, a barrier around the timed region and the max-over-ranks time; the whole-job rate is
the units of all ranks over the slowest rank's time (weak scaling)."""
from __future__ import annotations

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


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench.dist_env() == (ws, rank, rank)
        dist.barrier()
        local_seconds = 1.0 + rank          # rank 1 is the slow one
        t = bench.reduce_max_over_ranks(local_seconds, ws)
        rate = bench.whole_job_rate(100.0, t, ws)
        dist.barrier()
        q.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_rate():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, t, rate in res:
        assert t == pytest.approx(2.0)
        assert rate == pytest.approx(2 * 100.0 / 2.0)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10.0, 2.0, 1) == 5.0
