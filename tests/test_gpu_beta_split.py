"""The kernel-mode rounding correction of the mixed-precision 2-D operator (bn_options.beta_split).

In mixed precision the pair and triple sums read kernel-mode weights beta(a, b) (and the weights
formed from them) rounded to FP32.  That rounding is one fixed perturbation of the operator, so the
error it causes does not average out over the time steps of a run: it drives a drift of the mixed
state away from the FP64 one that grows linearly in time.  The correction runs the same FP32 kernels
a second time over tables of the rounding residuals x - fl32(x) and adds the result; Q^ is linear in
the weights, so the two passes together use the weights to about 48 bits.  The remaining FP32
roundings (of the modes, the products and the sums) change from step to step and largely average out.

The correction pays where the weight rounding dominates: at N = 16, whose inner sums are short.  At
N >= 32 the rounding of the long FP32 inner sums dominates instead, and the correction changes little
(measured on a stratified sample of the serving mix).

Checked here, through the C ABI: the correction cuts the drift of a run from the FP64 GPU run by a
large factor on two N = 16 requests of the seeded serving mix (one of which misses 1e-6 without it);
a standalone
evaluation with the correction stays within the mixed tolerance of the oracle and differs from the
uncorrected one by about the FP32 rounding of beta; the batched step, the server and the
no-allocation evaluation give bitwise the result of the solver alone.
"""
from __future__ import annotations

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


def _request(rid):
    return I.serving_requests(n=512, rate=200.0, Ns=(16, 32, 64), kernels=(0, 1))[rid]


def _run(B, r, steps, **opts):
    with B.Solver(2, r["N"], T6, r["R"], r["kernel"], r["eps"], **opts) as s:
        s.set_state(I.request_f0(r))
        s.step_rk(r["dt"], steps)
        return s.get_state()


# requests 181 (hard spheres, eps=-1, max f0 0.88) and 288 (hard spheres, eps=-1, max f0 0.47) of the
# seeded serving mix, N = 16, run to t = 2 (measured: 1.7e-6 -> 1.5e-7 and 4.6e-7 -> 8.1e-8)
@pytest.mark.parametrize("rid", [181, 288])
def test_correction_cuts_the_drift_from_fp64(B, rid):
    r = _request(rid)
    assert r["N"] == 16
    steps = int(round(r["t_end"] / r["dt"]))
    ref = _run(B, r, steps, precision=B.FP64)
    plain = _run(B, r, steps, precision=B.MIXED)
    split = _run(B, r, steps, precision=B.MIXED, beta_split=1)
    e_plain = np.linalg.norm(plain - ref) / np.linalg.norm(ref)
    e_split = np.linalg.norm(split - ref) / np.linalg.norm(ref)
    assert e_split <= e_plain / 3, (e_plain, e_split)
    assert e_split <= 3e-7, (e_plain, e_split)


@pytest.mark.parametrize("N,kernel,eps", [(16, 1, -1.0), (32, 0, 1.0), (64, 0, 1.0)])
def test_corrected_evaluation_parity(B, N, kernel, eps):
    f = I.two_gaussians(2, N, T6, 0.9, (1.2, 0.4), 0.85)
    with B.Solver(2, N, T6, R6, kernel, eps, precision=B.MIXED, beta_split=1) as s, \
            B.Solver(2, N, T6, R6, kernel, eps, precision=B.MIXED) as p:
        s.set_state(f)
        p.set_state(f)
        qs = s.eval_collision_modes()
        qp = p.eval_collision_modes()
        qs2 = s.eval_collision_modes()
    assert np.array_equal(qs, qs2)
    d = np.linalg.norm(qs - qp) / np.linalg.norm(qp)
    assert 1e-10 < d < 1e-6, d    # the correction is of the order of the FP32 rounding of beta
    op = O.Operator(2, N, T6, R6, kernel, eps)
    G = op.dft(f)
    if N <= 32:
        ref, gain = op.collision_modes(G)[:2]
        got = qs.reshape(N, N)
    else:   # N = 64: 4x4 blocks at a corner, on an edge, at the centre and at the opposite corner
        h = N // 2
        blocks = [(-h, -h), (-h, -2), (-2, -2), (h - 4, h - 4)]
        nl = np.array([(a + i, b + j) for a, b in blocks for i in range(4) for j in range(4)], dtype=np.int32)
        ref, gain = op.collision_modes_at(G, nl)[:2]
        got = qs.reshape(N, N)[nl[:, 0] + h, nl[:, 1] + h]
    err = np.linalg.norm(got - ref) / np.linalg.norm(gain)   # the mixed operator tolerance
    assert err <= 2e-6, err


def test_corrected_batch_and_server_equal_alone(B):
    mix = [(16, -1.0, 1), (32, 1.0, 1), (24, 1.0, 0), (64, -1.0, 1), (16, 0.0, 1)]
    dt, steps = 0.01, 3

    def f0(N, k):
        return I.two_gaussians(2, N, T6, 0.8 + 0.1 * k, (1.0 + 0.2 * k, 0.5), 0.5 + 0.05 * k)

    alone = []
    for k, (N, eps, bs) in enumerate(mix):
        with B.Solver(2, N, T6, R6, B.MAXWELL, eps, precision=B.MIXED, beta_split=bs) as s:
            s.set_state(f0(N, k))
            s.step_rk(dt, steps)
            alone.append(s.get_state())
    solvers = [B.Solver(2, N, T6, R6, B.MAXWELL, eps, precision=B.MIXED, beta_split=bs) for (N, eps, bs) in mix]
    for k, s in enumerate(solvers):
        s.set_state(f0(s.N, k))
    assert B.step_rk_batch(solvers, [dt] * len(solvers), steps) == -1
    for k, s in enumerate(solvers):
        assert np.array_equal(s.get_state(), alone[k]), k
        s.close()
    with B.Server(max_active=8) as srv:
        ids = [srv.submit(2, N, T6, R6, B.MAXWELL, eps, f0(N, k), dt, dt * steps, precision=B.MIXED, beta_split=bs)
               for k, (N, eps, bs) in enumerate(mix)]
        srv.wait_idle(300)
        for k, (N, _, _) in enumerate(mix):
            st, res, _ = srv.poll(ids[k], N * N)
            assert st == 2
            assert np.array_equal(res.reshape(N, N), alone[k].reshape(N, N)), k


def test_corrected_noalloc_equals_device_evaluation(B):
    torch = pytest.importorskip("torch")
    for N in (32, 64):
        with B.Solver(2, N, T6, R6, B.HARD_SPHERE, 1.0, precision=B.MIXED, beta_split=1) as s:
            f = I.two_gaussians(2, N, T6, 0.9, (1.5, -0.5), 0.8)
            f_dev = torch.tensor(f.reshape(-1), dtype=torch.float64, device="cuda")
            q_ref = torch.empty_like(f_dev)
            q_na = torch.full_like(f_dev, float("nan"))
            s.eval_collision_device(f_dev, q_ref)
            torch.cuda.synchronize()
            s.eval_collision_noalloc(f_dev, q_na, stream=torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert np.array_equal(q_na.cpu().numpy(), q_ref.cpu().numpy()), N


def test_beta_split_option_is_checked(B):
    with pytest.raises(B.BNError):
        B.Solver(2, 16, T6, R6, B.MAXWELL, 1.0, precision=B.MIXED, beta_split=2)
    # ignored in FP64: the FP64 kernels read the FP64 weights
    with B.Solver(2, 16, T6, R6, B.MAXWELL, 1.0, precision=B.FP64, beta_split=1) as s, \
            B.Solver(2, 16, T6, R6, B.MAXWELL, 1.0, precision=B.FP64) as p:
        f = I.two_gaussians(2, 16, T6, 0.9, (1.0, 0.5), 0.7)
        s.set_state(f)
        p.set_state(f)
        assert np.array_equal(s.eval_collision(), p.eval_collision())
