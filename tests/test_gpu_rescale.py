"""The velocity-rescaling method on the GPU (include/bn.h: bn_rescale_set, bn_step_rescaled) against
the FP64 oracle of the same procedure (oracle/rescaling.py; Mouton & Rey, Sec. 3.3, forward Euler).

Setup as in Sec. 4.1: the initial datum discretised on the velocity grid of scale 1 centred on its
mean gives the discrete mass, mean velocity and internal energy, hence the temperature (and fugacity)
and the scale w0 = sqrt(T0) (quantum) or sqrt(T0 + |u0|^2 / 2) (classical); G0 = (L / (pi w0))^2
f0(L xi / (pi w0) + u0) on the grid of [-pi, pi]^2, R = S = 2 pi / (3 + sqrt 2).  Several steps on both
sides; FP64: the state G and (w, u, rho, e) within 1e-12, mixed precision within 1e-6.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import rescaling as RS

pytestmark = pytest.mark.gpu

S_TRUNC = 2.0 * math.pi / (3.0 + math.sqrt(2.0))


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


def f0(v, amp):
    """Two Gaussian bumps (not an equilibrium), max below 1/|eps| for the quantum cases."""
    r1 = np.sum((v - [0.8, 0.3]) ** 2, -1)
    r2 = np.sum((v + [0.6, 0.5]) ** 2, -1)
    return amp * (np.exp(-r1 / 0.8) + 0.7 * np.exp(-r2 / 0.5))


def initial(N, L, eps, amp):
    j = np.arange(-N // 2, N // 2) * (2.0 * L / N)
    v = np.stack(np.meshgrid(j, j, indexing="ij"), -1)
    f = f0(v, amp)
    dv = (2.0 * L / N) ** 2
    rho = f.sum() * dv
    u = (v * f[..., None]).sum((0, 1)) * dv / rho
    # the grid of scale 1 centred on the discrete mean (Sec. 4.1, steps 2-3)
    vc = v + u
    fc = f0(vc, amp)
    rho = fc.sum() * dv
    e = 0.5 * (np.sum((vc - u) ** 2, -1) * fc).sum() * dv / rho
    T, _ = RS.temperature(2, eps, rho, e)
    w = RS.omega_of(2, eps, T, u)
    s = math.pi * w / L
    G = f0(u + RS.xi_grid(2, N) / s, amp) / s ** 2
    return G, rho, u, e, w


CASES = [  # (N, L, kernel, eps, amp, precision, tolerance, start off the scale)
    (16, 4.0, 0, -9.0, 0.06, "fp64", 1e-12, False),
    (16, 4.0, 0, -9.0, 0.06, "fp64", 1e-12, True),
    (16, 5.0, 0, 9.0, 0.01, "fp64", 1e-12, False),
    (16, 5.0, 0, 0.0, 0.3, "fp64", 1e-12, True),
    (12, 4.0, 1, -9.0, 0.06, "fp64", 1e-12, False),
    (16, 4.0, 0, -9.0, 0.06, "mixed", 1e-6, True),
]


@pytest.mark.parametrize("N,L,kernel,eps,amp,precision,tol,off", CASES)
def test_rescaled_steps_match_the_oracle(B, N, L, kernel, eps, amp, precision, tol, off):
    """`off`: the solve starts with w 25 % above sqrt(T) and u shifted, so that the first step moves
    the scale and the mean velocity by a lot and the divergence term carries real weight."""
    dt, steps = 0.01, 4
    G, rho, u, e, w = initial(N, L, eps, amp)
    if off:
        w, u = 1.25 * w, u + np.array([0.1, -0.05])
    run = RS.RescaledRun(N, L, S_TRUNC, kernel, eps, G, rho, u, e, w)
    for _ in range(steps):
        run.step(dt)
    prec = B.FP64 if precision == "fp64" else B.MIXED
    with B.Solver(2, N, math.pi, S_TRUNC, kernel, eps, precision=prec) as s:
        s.set_state(G)
        s.rescale_set(L, w, u, rho, e)
        s.step_rescaled(dt, steps)
        Gg = s.get_state().reshape(N, N)
        st = s.rescale_state()
    assert np.linalg.norm(Gg - run.G) <= tol * np.linalg.norm(run.G)
    assert st["w"] == pytest.approx(run.w, rel=tol)
    assert np.allclose(st["u"], run.u, rtol=tol, atol=tol * (abs(run.u).max() + w))
    assert st["rho"] == pytest.approx(run.rho, rel=tol) and st["e"] == pytest.approx(run.e, rel=tol)
    assert st["t"] == pytest.approx(steps * dt)
    assert w != run.w   # the scale moved: the divergence term was exercised


@pytest.mark.parametrize("N,L,kernel,eps,amp,off", [(16, 4.0, 0, -9.0, 0.06, True), (16, 5.0, 0, 0.0, 0.3, False),
                                                     (12, 4.0, 1, 9.0, 0.06, True)])
def test_rk2_rescaled_steps_match_the_oracle(B, N, L, kernel, eps, amp, off):
    """bn_step_rescaled_rk2 against the oracle's RK2 form (predictor, trapezoidal moments, midpoint
    rates; two evaluations per step): FP64 within 1e-12, several steps, on and off the scale."""
    dt, steps = 0.01, 3
    G, rho, u, e, w = initial(N, L, eps, amp)
    if off:
        w, u = 1.25 * w, u + np.array([0.1, -0.05])
    run = RS.RescaledRun(N, L, S_TRUNC, kernel, eps, G, rho, u, e, w)
    for _ in range(steps):
        run.step_rk2(dt)
    with B.Solver(2, N, math.pi, S_TRUNC, kernel, eps, precision=B.FP64) as s:
        s.set_state(G)
        s.rescale_set(L, w, u, rho, e)
        s.step_rescaled(dt, steps, rk2=True)
        Gg = s.get_state().reshape(N, N)
        st = s.rescale_state()
    assert np.linalg.norm(Gg - run.G) <= 1e-12 * np.linalg.norm(run.G)
    assert st["w"] == pytest.approx(run.w, rel=1e-12)
    assert np.allclose(st["u"], run.u, rtol=1e-12, atol=1e-12 * (abs(run.u).max() + w))
    assert st["rho"] == pytest.approx(run.rho, rel=1e-12) and st["e"] == pytest.approx(run.e, rel=1e-12)
    assert st["t"] == pytest.approx(steps * dt)


def test_rk2_rescaled_steps_3d(B):
    """3-D Fermi-Dirac hard spheres, N = 8, RK2 form, against the oracle (FP64, 1e-12)."""
    N, L, dt, steps, eps = 8, 4.0, 0.01, 2, -1.0
    j = np.arange(-N // 2, N // 2) * (2.0 * L / N)
    v = np.stack(np.meshgrid(j, j, j, indexing="ij"), -1)

    def g0(x):
        return 0.3 * np.exp(-np.sum((x - [0.5, 0.2, -0.1]) ** 2, -1) / 0.9) + \
            0.2 * np.exp(-np.sum((x + [0.4, 0.3, 0.0]) ** 2, -1) / 0.6)

    dv = (2.0 * L / N) ** 3
    f = g0(v)
    rho = f.sum() * dv
    u = (v * f[..., None]).sum((0, 1, 2)) * dv / rho
    e = 0.5 * (np.sum((v - u) ** 2, -1) * f).sum() * dv / rho
    T, _ = RS.temperature(3, eps, rho, e)
    w = 1.2 * RS.omega_of(3, eps, T, u)
    s = math.pi * w / L
    G = g0(u + RS.xi_grid(3, N) / s) / s ** 3
    run = RS.RescaledRun(N, L, S_TRUNC, 1, eps, G, rho, u, e, w, d=3, M1=4, M2=4)
    for _ in range(steps):
        run.step_rk2(dt)
    with B.Solver(3, N, math.pi, S_TRUNC, B.HARD_SPHERE, eps, precision=B.FP64, M1=4, M2=4) as sol:
        sol.set_state(G)
        sol.rescale_set(L, w, u, rho, e)
        sol.step_rescaled(dt, steps, rk2=True)
        Gg = sol.get_state().reshape((N,) * 3)
        st = sol.rescale_state()
    assert np.linalg.norm(Gg - run.G) <= 1e-12 * np.linalg.norm(run.G)
    assert st["w"] == pytest.approx(run.w, rel=1e-12) and st["z"] == pytest.approx(run.z, rel=1e-10)

@pytest.mark.parametrize("eps", [0.0, -1.0, 1.0])
def test_rescaled_steps_3d(B, eps):
    """3-D hard spheres, N = 8, started 20 % off the scale: eps = 0 (the classical temperature
    T = 2e/3), Fermi-Dirac and Bose-Einstein (x = 0.37: T and z from K_{3/2}, K_{5/2} by quadrature on
    both sides, the library's own double-exponential rule against the oracle's adaptive one)."""
    N, L, dt, steps = 8, 4.0, 0.01, 3
    j = np.arange(-N // 2, N // 2) * (2.0 * L / N)
    v = np.stack(np.meshgrid(j, j, j, indexing="ij"), -1)

    def g0(x):
        return 0.3 * np.exp(-np.sum((x - [0.5, 0.2, -0.1]) ** 2, -1) / 0.9) + \
            0.2 * np.exp(-np.sum((x + [0.4, 0.3, 0.0]) ** 2, -1) / 0.6)

    dv = (2.0 * L / N) ** 3
    f = g0(v)
    rho = f.sum() * dv
    u = (v * f[..., None]).sum((0, 1, 2)) * dv / rho
    e = 0.5 * (np.sum((v - u) ** 2, -1) * f).sum() * dv / rho
    T, _ = RS.temperature(3, eps, rho, e)
    w = 1.2 * RS.omega_of(3, eps, T, u)
    s = math.pi * w / L
    G = g0(u + RS.xi_grid(3, N) / s) / s ** 3
    run = RS.RescaledRun(N, L, S_TRUNC, 1, eps, G, rho, u, e, w, d=3, M1=4, M2=4)
    for _ in range(steps):
        run.step(dt)
    with B.Solver(3, N, math.pi, S_TRUNC, B.HARD_SPHERE, eps, precision=B.FP64, M1=4, M2=4) as sol:
        sol.set_state(G)
        sol.rescale_set(L, w, u, rho, e)
        sol.step_rescaled(dt, steps)
        Gg = sol.get_state().reshape((N,) * 3)
        st = sol.rescale_state()
    assert np.linalg.norm(Gg - run.G) <= 1e-12 * np.linalg.norm(run.G)
    assert st["w"] == pytest.approx(run.w, rel=1e-12) and np.allclose(st["u"], run.u, rtol=1e-12, atol=1e-13)
    assert st["rho"] == pytest.approx(run.rho, rel=1e-12) and st["e"] == pytest.approx(run.e, rel=1e-12)
    assert w != run.w
    if eps != 0.0:
        assert st["z"] == pytest.approx(run.z, rel=1e-10)
        with B.Solver(3, N, math.pi, S_TRUNC, B.HARD_SPHERE, eps, M1=4, M2=4) as sol:
            # moments beyond the end of I_eq (x = 1.001 times it): degenerate / condensed
            xmax = RS.IEQ_FD_3D if eps < 0 else RS.IEQ_BE_3D
            e_out = 0.75 * (1.0 / (1.001 * xmax)) ** (2.0 / 3.0) / math.pi
            with pytest.raises(B.BNError) as ei:
                sol.rescale_set(L, 1.0, [0.0, 0.0, 0.0], 1.0, e_out)
            assert ei.value.status == -7


def test_rescaling_arguments_and_degenerate_state(B):
    with B.Solver(2, 16, 4.0, 1.0, 0, -9.0) as s:
        with pytest.raises(B.BNError) as ei:          # the box must be T = pi
            s.rescale_set(4.0, 1.0, [0.0, 0.0], 1.0, 1.0)
        assert ei.value.status == -1
    with B.Solver(2, 16, math.pi, S_TRUNC, 0, -9.0) as s:
        s.set_state(np.full((16, 16), 0.01))
        with pytest.raises(B.BNError) as ei:
            s.step_rescaled(0.01, 1)                  # before bn_rescale_set
        assert ei.value.status == -7
        with pytest.raises(B.BNError) as ei:          # 2-D Fermi-Dirac: |eps| rho / (2 pi e) >= 2
            s.rescale_set(4.0, 1.0, [0.0, 0.0], 1.0, 9.0 / (2 * math.pi * 2.5))
        assert ei.value.status == -7
