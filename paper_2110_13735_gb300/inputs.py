"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle's tests.

This module holds initial data only -- no arithmetic of the collision operator.
Every workload is an analytic initial datum of the kind used in Mouton & Rey,
arXiv:2110.13735 (Gaussians, two-Gaussian mixtures, quantum Maxwellians of
Sec. 1.2) or the 2-D Maxwell-molecule BKW solution (Bobylev; Krook & Wu), all
sampled on the grid v_j = 2Tj/N, j in I_N = {-N/2..N/2-1}^d (Sec. 3.3).
Seeds come from numpy's PCG64 with base seed 211013735.
"""
from __future__ import annotations

import math

import numpy as np

SEED = 211013735


def box_half_width(R: float) -> float:
    """T = (3+sqrt 2) R / 2: the box for which R_xi = pi R / T = 2 pi/(3+sqrt 2) (Sec. 4.1)."""
    return (3.0 + math.sqrt(2.0)) * R / 2.0


def grid(d: int, N: int, T: float) -> np.ndarray:
    """Grid velocities v_j = 2Tj/N, shape (N,)*d + (d,), row-major, last axis fastest."""
    j = np.arange(-N // 2, N // 2, dtype=np.float64) * (2.0 * T / N)
    return np.stack(np.meshgrid(*([j] * d), indexing="ij"), axis=-1)


def gaussian(d: int, N: int, T: float, rho: float, temp: float, u=None) -> np.ndarray:
    """rho (2 pi temp)^{-d/2} exp(-|v-u|^2/(2 temp))."""
    v = grid(d, N, T)
    u = np.zeros(d) if u is None else np.asarray(u, float)
    r2 = np.sum((v - u) ** 2, axis=-1)
    return rho * (2.0 * math.pi * temp) ** (-d / 2.0) * np.exp(-r2 / (2.0 * temp))


def _two_gauss_profile(v, c, sigma):
    return np.exp(-np.sum((v - c) ** 2, -1) / (2 * sigma)) + np.exp(-np.sum((v + c) ** 2, -1) / (2 * sigma))


def two_gaussians_amplitude(c, sigma: float, fmax: float) -> float:
    """Amplitude A with max_v A[g(v-c)+g(v+c)] = fmax, g = exp(-|v|^2/(2 sigma)).

    The maximum of the symmetric pair lies on the segment between the centres;
    it is found by a dense 1-D search refined by golden section.
    """
    c = np.asarray(c, float)
    s = np.linspace(0.0, 1.5, 20001)
    vals = _two_gauss_profile(s[:, None] * c[None, :], c, sigma)
    i = int(np.argmax(vals))
    lo, hi = s[max(i - 1, 0)], s[min(i + 1, s.size - 1)]
    g = (math.sqrt(5) - 1) / 2
    for _ in range(200):
        a = hi - g * (hi - lo)
        b = lo + g * (hi - lo)
        fa = _two_gauss_profile((a * c)[None, :], c, sigma)[0]
        fb = _two_gauss_profile((b * c)[None, :], c, sigma)[0]
        if fa < fb:
            lo = a
        else:
            hi = b
    peak = _two_gauss_profile((0.5 * (lo + hi) * c)[None, :], c, sigma)[0]
    return fmax / peak


def two_gaussians(d: int, N: int, T: float, sigma: float, centre, fmax: float) -> np.ndarray:
    """A[g(v-c)+g(v+c)] with sigma the variance (temperature) and max over R^d equal to fmax."""
    c = np.asarray(centre, float)
    A = two_gaussians_amplitude(c, sigma, fmax)
    return A * _two_gauss_profile(grid(d, N, T), c, sigma)


def bkw_2d(t: float, v: np.ndarray) -> np.ndarray:
    """2-D BKW solution for Maxwell molecules with B = 1/(2 pi):
    f = (2 pi K^2)^-1 exp(-|v|^2/(2K)) (2K - 1 + (1-K)|v|^2/(2K)), K = 1 - exp(-t/8)/2."""
    K = 1.0 - 0.5 * math.exp(-t / 8.0)
    r2 = np.sum(v * v, axis=-1)
    return np.exp(-r2 / (2 * K)) / (2 * math.pi * K * K) * (2 * K - 1 + (1 - K) * r2 / (2 * K))


def bkw_2d_dt(t: float, v: np.ndarray) -> np.ndarray:
    """d/dt of :func:`bkw_2d` (chain rule through K(t))."""
    K = 1.0 - 0.5 * math.exp(-t / 8.0)
    dK = 0.5 * math.exp(-t / 8.0) / 8.0
    r2 = np.sum(v * v, axis=-1)
    E = np.exp(-r2 / (2 * K))
    A = 1.0 / (2 * math.pi * K * K)
    Bq = 2 * K - 1 + (1 - K) * r2 / (2 * K)
    dA = -2.0 / (2 * math.pi * K ** 3)
    dE = E * r2 / (2 * K * K)
    dB = 2 - r2 / (2 * K * K)
    return (dA * E * Bq + A * dE * Bq + A * E * dB) * dK


def config0_f0(N: int = 16, R: float = 6.0) -> np.ndarray:
    """2-D Fermi-Dirac workload: two isotropic Gaussians (sigma=1, centres +-(2,1)), max 0.8."""
    return two_gaussians(2, N, box_half_width(R), 1.0, (2.0, 1.0), 0.8)


def config1_bkw_f0(N: int = 32, R: float = 6.0, t0: float = 1.0) -> np.ndarray:
    """2-D classical workload: the BKW datum at t0."""
    return bkw_2d(t0, grid(2, N, box_half_width(R)))


def config1_boson_f0(N: int = 32, R: float = 6.0) -> np.ndarray:
    """2-D bosonic workload: a Gaussian of mass 5 and temperature 0.5."""
    return gaussian(2, N, box_half_width(R), 5.0, 0.5)


def config2_f0(N: int = 32, R: float = 6.0) -> np.ndarray:
    """3-D Fermi-Dirac workload: two Gaussians (variance 0.8, centres +-(1.5,0,0)), max 0.9."""
    return two_gaussians(3, N, box_half_width(R), 0.8, (1.5, 0.0, 0.0), 0.9)


def config4_f0(N: int = 48, R: float = 6.0) -> np.ndarray:
    """3-D bosonic workload: a Gaussian of mass 8 and temperature 0.4."""
    return gaussian(3, N, box_half_width(R), 8.0, 0.4)


def serving_requests(n: int = 512, seed: int = SEED, rate: float = 200.0, t_end: float = 2.0,
                     dt: float = 0.01, Ns=(16, 32, 64), kernels=(0,)):
    """The serving mix: n 2-D requests with N ~ U(Ns), eps ~ U{-1,0,+1}, kernel ~ U(kernels),
    sigma ~ U[0.5,1.5], centres +-c with c uniform in the disk of radius 2.5,
    max f0 ~ U[0.1,0.9], Poisson arrivals at ``rate`` per second."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(n):
        N = int(rng.choice(Ns))
        eps = float(rng.choice([-1.0, 0.0, 1.0]))
        kernel = int(rng.choice(kernels))
        sigma = float(rng.uniform(0.5, 1.5))
        rad = 2.5 * math.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * math.pi)
        c = (rad * math.cos(ang), rad * math.sin(ang))
        fmax = float(rng.uniform(0.1, 0.9))
        reqs.append(dict(id=i, arrival=float(arrivals[i]), N=N, eps=eps, kernel=kernel, sigma=sigma,
                         centre=c, fmax=fmax, R=6.0, dt=dt, t_end=t_end))
    return reqs


def request_f0(req) -> np.ndarray:
    T = box_half_width(req["R"])
    return two_gaussians(2, req["N"], T, req["sigma"], req["centre"], req["fmax"])
