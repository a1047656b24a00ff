"""Host-side equilibrium builders used as test fixtures (Mouton & Rey, Sec. 1.2).

Quantum Maxwellian (def_Mq_2d): M_q(v) = (1/|alpha|) / (z^{-1} exp(|v-u|^2/(2T)) + sgn(alpha)),
alpha = +hbar^d (Fermi-Dirac), -hbar^d (Bose-Einstein).  Its mass is
rho = (2 pi T)^{d/2} K_{d/2}(z) / |alpha| (mom02_qmaxwell) with K = F (Fermi-Dirac
integral, = -Li_nu(-z)) or B (Bose-Einstein integral, = Li_nu(z)).  The fugacity
is found with Brent's method as the paper does (Sec. 1.2, practical computations).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize, special


def fd_integral(nu: float, z: float) -> float:
    """F_nu(z) = Gamma(nu)^-1 int_0^inf x^{nu-1} / (z^-1 e^x + 1) dx."""
    if nu == 1.0:
        return math.log1p(z)
    f = lambda x: x ** (nu - 1.0) * z * math.exp(-x) / (1.0 + z * math.exp(-x))
    val, _ = integrate.quad(f, 0.0, math.inf, epsabs=0, epsrel=1e-13, limit=400)
    return val / special.gamma(nu)


def be_integral(nu: float, z: float) -> float:
    """B_nu(z) = Gamma(nu)^-1 int_0^inf x^{nu-1} / (z^-1 e^x - 1) dx, 0 < z < 1."""
    if nu == 1.0:
        return -math.log1p(-z)
    f = lambda x: x ** (nu - 1.0) * z * math.exp(-x) / (1.0 - z * math.exp(-x))
    val, _ = integrate.quad(f, 0.0, math.inf, epsabs=0, epsrel=1e-13, limit=400)
    return val / special.gamma(nu)


def mass(d: int, stat: str, z: float, temp: float, abs_alpha: float) -> float:
    K = fd_integral(d / 2.0, z) if stat == "FD" else be_integral(d / 2.0, z)
    return (2.0 * math.pi * temp) ** (d / 2.0) * K / abs_alpha


def fugacity(d: int, stat: str, rho: float, temp: float, abs_alpha: float) -> float:
    """Brent on mu = ln z for Fermi-Dirac, on z for Bose-Einstein (Sec. 1.2)."""
    if stat == "FD":
        g = lambda mu: mass(d, "FD", math.exp(mu), temp, abs_alpha) - rho
        return math.exp(optimize.brentq(g, -50.0, 50.0, xtol=1e-15, rtol=1e-15))
    g = lambda z: mass(d, "BE", z, temp, abs_alpha) - rho
    return optimize.brentq(g, 1e-14, 1.0 - 1e-15, xtol=1e-16, rtol=1e-15)


def quantum_maxwellian(v: np.ndarray, stat: str, z: float, temp: float, abs_alpha: float, u=None) -> np.ndarray:
    u = np.zeros(v.shape[-1]) if u is None else np.asarray(u, float)
    r2 = np.sum((v - u) ** 2, axis=-1)
    s = 1.0 if stat == "FD" else -1.0
    return (1.0 / abs_alpha) / (np.exp(r2 / (2.0 * temp)) / z + s)
