"""Pins of the oracle's moments (E_c, H) and of its conservation projection.

* E_c and H of a Gaussian and of a quantum Maxwellian against closed forms.  For the
  quantum Maxwellian f = u / (alpha (1 + u)), u = s z exp(-|v|^2/(2T)), alpha = s |alpha|
  (s = +1 Fermi-Dirac, -1 Bose-Einstein; Sec. 1.2, def_Mq_2d), one has 1 - alpha f = 1/(1+u) and
  f ln f + (1 - alpha f)/alpha ln(1 - alpha f) = f (ln z - ln|alpha| - |v|^2/(2T)) - ln(1+u)/alpha,
  whose integral is, with K = F (Fermi-Dirac) or B (Bose-Einstein) of Sec. 1.2,
      H   = rho ln(z/|alpha|) - (d/2 + 1) (2 pi T)^{d/2} K_{d/2+1}(z) / |alpha|,
      E_c = d T (2 pi T)^{d/2} K_{d/2+1}(z) / |alpha|,   rho = (2 pi T)^{d/2} K_{d/2}(z) / |alpha|.
  (The classical limit z -> 0 gives rho ln(rho/(2 pi T)^{d/2}) - (d/2 + 1) rho: the Gaussian's
  f ln f entropy minus rho from the (1 - alpha f)/alpha ln(1 - alpha f) term.)  A sign slip in
  that term moves H by about 2 rho.
* The projection Q - C^T (C C^T)^{-1} C Q (C: the invariants 1, v, |v|^2 on the grid) is the
  orthogonal projector onto the grid functions with zero mass, momentum and energy: it maps
  every invariant to zero, leaves every function orthogonal to them unchanged, and is
  idempotent; these three facts determine it.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
from paper_2110_13735_gb300 import inputs as I
from tests import equilibria as EQ


def test_Ec_and_H_of_a_gaussian_classical():
    """eps = 0: E_c = rho (d T + |u|^2), H = rho ln(rho/(2 pi T)^{d/2}) - d rho / 2."""
    for d, N in ((2, 32), (3, 24)):
        L = 9.0
        op = O.Operator(d, N, L, 2 * L / (3 + math.sqrt(2)), 0 if d == 2 else 1, 0.0)
        rho, temp = 1.7, 0.9
        u = np.array([0.4, -0.3, 0.2][:d])
        f = I.gaussian(d, N, L, rho, temp, u=u)
        m = op.moments(f)
        Ec, H = m[d + 2], m[d + 3]
        assert Ec == pytest.approx(rho * (d * temp + float(u @ u)), rel=1e-9)
        assert H == pytest.approx(rho * math.log(rho / (2 * math.pi * temp) ** (d / 2)) - d * rho / 2, rel=1e-9)


@pytest.mark.parametrize("d,stat,sig", [(2, "FD", 1.0), (2, "BE", 1.0), (3, "FD", 1.0), (2, "FD", 0.5)])
def test_Ec_and_H_of_a_quantum_maxwellian(d, stat, sig):
    hbar = 3.0
    aa = hbar ** d
    alpha = aa if stat == "FD" else -aa
    N, L = (96, 8.0) if d == 2 else (32, 8.0)   # the Bose-Einstein integrand has poles 0.74 from the real axis
    z = EQ.fugacity(d, stat, 1.0, sig, aa)
    op = O.Operator(d, N, L, 2 * L / (3 + math.sqrt(2)), 0 if d == 2 else 1, -alpha)
    f = EQ.quantum_maxwellian(op.velocities(), stat, z, sig, aa)
    m = op.moments(f)
    K = EQ.fd_integral if stat == "FD" else EQ.be_integral
    c = (2 * math.pi * sig) ** (d / 2) / aa
    rho = c * K(d / 2, z)
    Ec = d * sig * c * K(d / 2 + 1, z)
    H = rho * math.log(z / aa) - (d / 2 + 1) * c * K(d / 2 + 1, z)
    assert m[0] == pytest.approx(rho, rel=1e-7)
    assert m[d + 2] == pytest.approx(Ec, rel=1e-7)
    assert m[d + 3] == pytest.approx(H, rel=1e-7, abs=1e-9)


def _invariants(op):
    v = op.velocities().reshape(-1, op.d)
    return np.concatenate([np.ones((v.shape[0], 1)), v, np.sum(v * v, axis=1, keepdims=True)], axis=1)


@pytest.mark.parametrize("d,N", [(2, 16), (3, 8)])
def test_conservation_projection_is_the_orthogonal_projector(d, N):
    op = O.Operator(d, N, 13.0, 6.0, 0 if d == 2 else 1, 1.0)
    C = _invariants(op)                     # (n, d+2)
    rng = np.random.default_rng(3 + d)
    Q = rng.standard_normal(op.n_modes)
    PQ = op.conserve(Q).reshape(-1)
    # the invariants of the result vanish (to rounding of the large |v|^2 column)
    assert np.abs(C.T @ PQ).max() <= 1e-10 * np.abs(C).max() * np.abs(Q).sum()
    # every invariant is mapped to zero
    for c in range(d + 2):
        col = C[:, c]
        assert np.abs(op.conserve(col).reshape(-1)).max() <= 1e-10 * np.abs(col).max()
    # a function orthogonal to the invariants is unchanged
    W = rng.standard_normal(op.n_modes)
    W -= C @ np.linalg.lstsq(C, W, rcond=None)[0]
    assert np.abs(op.conserve(W).reshape(-1) - W).max() <= 1e-10 * np.abs(W).max()
    # idempotent
    assert np.abs(op.conserve(PQ).reshape(-1) - PQ).max() <= 1e-10 * np.abs(PQ).max()
