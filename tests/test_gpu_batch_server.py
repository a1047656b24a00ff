"""Batched stepping (shared launches) and the continuous-batching server, through the C ABI.

A request advanced inside a batch, or inside the server among other requests, must give the same
result as alone (bitwise: every request keeps its own CTA partition and reduction order), and the
server's results match the FP64 oracle."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle as O
from paper_2110_13735_gb300 import inputs as I

pytestmark = pytest.mark.gpu

R6 = 6.0
T6 = I.box_half_width(R6)


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_13735_gb300 import build as BUILD
    BUILD.build()
    from paper_2110_13735_gb300 import bn
    bn.load()
    return bn


MIX = [  # (N, eps, precision)
    (16, -1.0, "mixed"), (32, 1.0, "fp64"), (16, 0.0, "fp64"), (24, 2.5, "mixed"), (64, 1.0, "mixed"),
    (32, -1.0, "mixed"),
]


def _f0(N, k):
    return I.two_gaussians(2, N, T6, 0.8 + 0.1 * k, (1.0 + 0.2 * k, 0.5), 0.5 + 0.05 * k)


def _prec(B, p):
    return B.MIXED if p == "mixed" else B.FP64


def test_batch_equals_alone(B):
    steps, dt = 3, 0.01
    alone = []
    for k, (N, eps, p) in enumerate(MIX):
        with B.Solver(2, N, T6, R6, B.MAXWELL, eps, precision=_prec(B, p)) as s:
            s.set_state(_f0(N, k))
            s.step_rk(dt, steps)
            alone.append(s.get_state())
    solvers = [B.Solver(2, N, T6, R6, B.MAXWELL, eps, precision=_prec(B, p)) for (N, eps, p) in MIX]
    for k, s in enumerate(solvers):
        s.set_state(_f0(s.N, k))
    assert B.step_rk_batch(solvers, [dt] * len(solvers), steps) == -1
    for k, s in enumerate(solvers):
        got = s.get_state()
        assert np.array_equal(got, alone[k]), (k, np.abs(got - alone[k]).max())
        assert s.moments()[-1] == pytest.approx(steps * dt)
        s.close()


def test_server_alone_vs_mix_and_oracle(B):
    N, eps, dt, t_end = 16, -1.0, 0.01, 0.05
    f0 = I.config0_f0(N)
    with B.Server(max_active=16) as srv:
        rid = srv.submit(2, N, T6, R6, B.MAXWELL, eps, f0, dt, t_end)
        srv.wait_idle(300)
        st, alone, times = srv.poll(rid, N * N)
        assert st == 2 and times[2] >= times[1] >= times[0]
    with B.Server(max_active=16) as srv:
        ids = []
        for k, (Nk, ek, p) in enumerate(MIX):
            ids.append(srv.submit(2, Nk, T6, R6, B.MAXWELL, ek, _f0(Nk, k), 0.01, 0.03 + 0.01 * k,
                                  precision=_prec(B, p)))
        rid = srv.submit(2, N, T6, R6, B.MAXWELL, eps, f0, dt, t_end)
        srv.wait_idle(600)
        st, mixed, _ = srv.poll(rid, N * N)
        assert st == 2
        for i in ids:
            assert srv.poll(i)[0] == 2
        stats = srv.stats()
        assert stats["done"] == len(MIX) + 1 and stats["failed"] == 0
    assert np.array_equal(alone.reshape(N, N), mixed.reshape(N, N))
    ora = O.Operator(2, N, T6, R6, 0, eps, M=2 * N)
    f_o = ora.step(f0, dt, int(round(t_end / dt)), 0)
    assert np.linalg.norm(alone.reshape(N, N) - f_o) / np.linalg.norm(f_o) <= 1e-12


def test_server_admission_by_memory(B):
    """With a budget for one operator's tables plus two solvers, at most two requests run at once
    and every request still completes."""
    N = 16
    nExt, nm, P = 4 * N * N, N * N, 2 * N
    # alpha tables; beta in FP64, FP32 and its FP32 residuals; the reducible (FP64, FP32, residual) and
    # quadratic (FP32, residual) weights; the transposed FP32 table and its residuals (N <= 32)
    tables = 2 * P * nExt * 8 + nExt * nExt * 16 + nExt * nm * 24 + 2 * nExt * nExt * 4
    solver = nm * (6 * 8 + 7 * 16 + 8) + nExt * 16 + 152 * 4 * nm * 16 + (1 << 16)
    with B.Server(device_bytes=tables + 2 * solver + 1024, max_active=16) as srv:
        ids = [srv.submit(2, N, T6, R6, B.MAXWELL, 1.0, _f0(N, k), 0.01, 0.02) for k in range(5)]
        srv.wait_idle(300)
        assert all(srv.poll(i)[0] == 2 for i in ids)
        st = srv.stats()
        assert st["max_active"] <= 2 and st["done"] == 5


def test_server_admits_least_work_first(B):
    """With one slot busy, of two queued requests the one with less estimated work (steps x terms
    per evaluation) is admitted first, whatever the submission order."""
    with B.Server(max_active=1) as srv:
        blocker = srv.submit(2, 16, T6, R6, B.MAXWELL, 1.0, _f0(16, 0), 0.01, 1.0)   # 100 steps
        deadline = time.monotonic() + 60
        while srv.poll(blocker)[0] == 0 and time.monotonic() < deadline:
            time.sleep(0.001)
        assert srv.poll(blocker)[0] >= 1
        big = srv.submit(2, 32, T6, R6, B.MAXWELL, 1.0, _f0(32, 1), 0.01, 0.05)
        small = srv.submit(2, 16, T6, R6, B.MAXWELL, 0.0, _f0(16, 2), 0.01, 0.05)
        srv.wait_idle(300)
        t_blk, t_big, t_small = (srv.poll(i)[2] for i in (blocker, big, small))
        assert all(srv.poll(i)[0] == 2 for i in (blocker, big, small))
    assert t_small[1] <= t_big[1]      # admission times
    assert t_small[1] >= t_blk[1]


def test_server_failed_request(B):
    """A request the library rejects (box too small for R: the anti-aliasing condition fails at
    solver creation) fails alone; the others complete."""
    with B.Server(max_active=4) as srv:
        bad = srv.submit(2, 16, 13.0, R6, B.MAXWELL, 1.0, _f0(16, 0), 0.01, 0.02)
        good = srv.submit(2, 16, T6, R6, B.MAXWELL, 1.0, _f0(16, 0), 0.01, 0.02)
        srv.wait_idle(300)
        assert srv.poll(bad)[0] == 3
        assert srv.poll(good)[0] == 2
