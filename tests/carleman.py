"""Direct quadrature of the truncated Carleman integral (Mouton & Rey, Sec. 2.2,
the FHJ truncation eq. IndicatorFilbetHuJin) for a band-limited G -- an
independent check of the oracle's Fourier-Galerkin sums (Lemma of Sec. 2.3).

For G(eta) = sum_k Ghat_k e^{i k.eta} (k in I_N, complex coefficients allowed:
every sub-operator is multilinear), the truncated operator is

  Q^R_alpha(G)(xi) = int_{B_R^2} Btilde delta(x.y) [G(xi+x)G(xi+y)(1 - alpha(G(xi)+G(xi+x+y)))
                     - G(xi)G(xi+x+y)(1 - alpha(G(xi+x)+G(xi+y)))] dx dy.

The delta is resolved by parametrising x and the hyperplane orthogonal to it:
  2-D: x = rho e_t, y = rho' e_{t+pi/2}: int_0^pi dt int_{-R}^{R} drho int_{-R}^{R} drho'
  3-D: x = rho e (e on a half sphere), y in the disk of radius R orthogonal to e:
       int_{S2+} de int_{-R}^{R} |rho| drho int_0^R r dr int_0^{2pi} dphi.
No part of this file is shared with the oracle or with the CUDA path.
"""
from __future__ import annotations

import numpy as np


def _modes(d, N):
    ks = np.arange(-N // 2, N // 2)
    return np.stack(np.meshgrid(*([ks] * d), indexing="ij"), axis=-1).reshape(-1, d).astype(np.float64)


def _integrand(G0, G1, G2, G3, alpha):
    return G1 * G2 * (1.0 - alpha * (G0 + G3)) - G0 * G3 * (1.0 - alpha * (G1 + G2))


def carleman_2d(Ghat, N, R, Btilde, alpha, xi, n_theta=128, n_rho=48):
    """``Btilde`` is a constant (Maxwell molecules) or a function of (|x|, |y|) on the node grid
    (hard spheres: 2 C_Phi sqrt(|x|^2 + |y|^2))."""
    K = _modes(2, N)
    g = np.asarray(Ghat).reshape(-1) * np.exp(1j * (K @ np.asarray(xi, float)))
    G0 = g.sum()
    x, w = np.polynomial.legendre.leggauss(n_rho)
    rho, wr = R * x, R * w
    Bw = Btilde(np.abs(rho)[:, None], np.abs(rho)[None, :]) if callable(Btilde) else Btilde
    total = 0.0 + 0.0j
    for t in np.arange(n_theta) * np.pi / n_theta:
        e = np.array([np.cos(t), np.sin(t)])
        ep = np.array([-np.sin(t), np.cos(t)])
        A = np.exp(1j * np.outer(rho, K @ e))
        B = np.exp(1j * np.outer(rho, K @ ep))
        G1 = (A @ g)[:, None]
        G2 = (B @ g)[None, :]
        G3 = (A[:, None, :] * B[None, :, :]) @ g
        total += wr @ (Bw * _integrand(G0, G1, G2, G3, alpha)) @ wr
    return (np.pi / n_theta) * total


def carleman_3d(Ghat, N, R, Btilde, alpha, xi, n_mu=16, n_phi=32, n_rho=12, n_r=12, n_t=32):
    K = _modes(3, N)
    g = np.asarray(Ghat).reshape(-1) * np.exp(1j * (K @ np.asarray(xi, float)))
    G0 = g.sum()
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    xr, wr_ = np.polynomial.legendre.leggauss(n_rho)
    rp = 0.5 * R * (xr + 1.0)
    wp = 0.5 * R * wr_
    rho = np.concatenate([-rp, rp])
    wrho = np.concatenate([wp, wp]) * np.abs(rho)
    xq, wq = np.polynomial.legendre.leggauss(n_r)
    r = 0.5 * R * (xq + 1.0)
    w_r = 0.5 * R * wq * r
    tt = np.arange(n_t) * 2.0 * np.pi / n_t
    wdisk = (w_r[:, None] * (2.0 * np.pi / n_t) * np.ones(n_t)[None, :]).reshape(-1)
    total = 0.0 + 0.0j
    for im, m in enumerate(mu):
        st = np.sqrt(max(0.0, 1.0 - m * m))
        for ph in np.arange(n_phi) * np.pi / n_phi:
            e = np.array([st * np.cos(ph), st * np.sin(ph), m])
            a = np.array([1.0, 0.0, 0.0]) if abs(e[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
            u = a - (a @ e) * e
            u /= np.linalg.norm(u)
            w = np.cross(e, u)
            A = np.exp(1j * np.outer(rho, K @ e))
            dirs = np.cos(tt)[:, None] * u[None, :] + np.sin(tt)[:, None] * w[None, :]
            Y = (r[:, None, None] * dirs[None, :, :]).reshape(-1, 3)
            B = np.exp(1j * (Y @ K.T))
            G1 = (A @ g)[:, None]
            G2 = (B @ g)[None, :]
            G3 = (A[:, None, :] * B[None, :, :]) @ g
            total += wmu[im] * (np.pi / n_phi) * (wrho @ _integrand(G0, G1, G2, G3, alpha) @ wdisk)
    return Btilde * total
