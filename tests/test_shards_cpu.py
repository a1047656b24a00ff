"""One 3-D evaluation split over ranks by output planes (the partition of bn_plan_shards), tested
on CPU ranks (gloo, world size 2) with the FP64 oracle as the evaluator of each shard.

Every output mode n of the Lemma of Sec. 2.3 depends on the whole of G^ but on no other output, so
the output planes n_0 can be split across GPUs, each holding the replicated G^ (at most 1.8 MB), and
one all-reduce (a sum of N^d complex values, the shards being zero outside their planes) assembles
Q^ for the next Runge-Kutta stage.  Checked here: the partition covers the planes of I_N once, in
contiguous ranges of nearly equal Q_{1,q} work; and the gathered shards are exactly the one-rank
result (each output is computed by the same oracle arithmetic; the all-reduce only adds zeros).
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2110_13735_gb300 import bn  # noqa: E402
from paper_2110_13735_gb300 import build as BUILD  # noqa: E402


def _plane_weights(N, wrap):
    """Q_{1,q} terms of each output plane n_0 (up to a common factor): the number of (k, l, m) in
    I_N^3 with k + l + m = n_0 (LINEAR) or = n_0 mod N (CIRCULAR), by enumeration."""
    I = np.arange(-N // 2, N // 2)
    s = (I[:, None, None] + I[None, :, None] + I[None, None, :]).ravel()
    if wrap:
        s = (s + N // 2) % N - N // 2
    return np.array([np.sum(s == n) for n in I], dtype=float)


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return bn.load()


@pytest.mark.parametrize("N,count,wrap", [(8, 2, 0), (16, 3, 0), (32, 4, 0), (48, 8, 0), (16, 3, 1), (32, 5, 1)])
def test_partition_covers_the_planes_once_and_balances_the_work(lib, N, count, wrap):
    b = bn.plan_shards(3, N, count, wrap=wrap)
    assert b[0] == 0 and b[-1] == N and np.all(np.diff(b) >= 1)
    w = _plane_weights(N, wrap)
    share = w.sum() / count
    loads = np.array([w[b[r]:b[r + 1]].sum() for r in range(count)])
    assert loads.sum() == pytest.approx(w.sum())
    # contiguous shards of whole planes: no shard exceeds its share by more than one plane
    assert loads.max() <= share + w.max()


def test_plan_shards_rejects_bad_arguments(lib):
    for args in [(2, 16, 0, 2), (3, 15, 0, 2), (3, 16, 0, 0), (3, 16, 0, 17), (3, 16, 2, 2)]:
        out = np.zeros(20, dtype=np.int32)
        import ctypes
        st = lib.bn_plan_shards(*args, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), out.size)
        assert st == -1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


N_SH, EPS = 6, 1.0


def _state():
    from paper_2110_13735_gb300 import inputs as I
    T = I.box_half_width(6.0)
    rng = np.random.Generator(np.random.PCG64(I.SEED + 77))
    f = I.two_gaussians(3, N_SH, T, 0.9, (1.5, 0.0, 0.0), 0.8) * (1.0 + 0.2 * rng.uniform(size=(N_SH,) * 3))
    return T, f


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        O.set_threads(2)
        T, f = _state()
        op = O.Operator(3, N_SH, T, 6.0, 1, EPS, M1=4, M2=4)
        G = op.dft(f)
        b = bn.plan_shards(3, N_SH, ws)
        h = N_SH // 2
        planes = range(b[rank], b[rank + 1])
        nl = np.array([(p - h, i - h, j - h) for p in planes for i in range(N_SH) for j in range(N_SH)],
                      dtype=np.int32)
        Qs = op.collision_modes_at(G, nl)[0]
        full = np.zeros((N_SH,) * 3, complex)
        for n, v in zip(nl, Qs):
            full[tuple(n + h)] = v
        t = torch.from_numpy(full.view(np.float64).copy())
        dist.all_reduce(t)          # the one collective of a sharded stage
        q.put((rank, t.numpy().view(np.complex128).reshape((N_SH,) * 3)))
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_gather_to_the_one_rank_result(lib):
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(ws))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    import oracle as O
    T, f = _state()
    op = O.Operator(3, N_SH, T, 6.0, 1, EPS, M1=4, M2=4)
    h = N_SH // 2
    nl = np.array([(p - h, i - h, j - h) for p in range(N_SH) for i in range(N_SH) for j in range(N_SH)], dtype=np.int32)
    ref = op.collision_modes_at(op.dft(f), nl)[0].reshape((N_SH,) * 3)
    for r in range(ws):
        assert np.array_equal(got[r], ref)
    # and the same as the oracle's table path to its rounding
    tab = op.collision_modes(op.dft(f))[0]
    assert np.abs(ref - tab).max() <= 1e-13 * np.abs(tab).max()
