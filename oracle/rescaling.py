"""FP64 CPU oracle of the velocity-rescaling method (Mouton & Rey, Sec. 3), 2-D and 3-D.

TEST INFRASTRUCTURE ONLY, like the rest of this package: the product library never imports it.

The rescaled unknown G lives on the grid xi_j = 2 pi j / N, j in I_N, of [-pi, pi]^d, and
f(t, v) = (pi w / L)^d G(t, (pi w / L)(v - u)) (eq. rescaling_def_fg with mu = 1, lambda = 1, the
velocity rescaling method of Sec. 3.2).  The collision operator transforms as
Q_eps(f)(v) = (pi w / L)^{d - gamma} Q_{eps (pi w / L)^d}(G)(xi) (eq. rescaling_collision; eps = -alpha,
the quantum parameter of this project), so the operator of G is the one of this package's
``Operator`` on the box T = pi with the kernel truncation R and eps_eff = eps (pi w / L)^d.

One step follows the numbered procedure of Sec. 3.3 for the forward Euler scheme, in its order:
  1. the state: G^n, rho^n, u^n, e^n, w^n;
  2. Q^n = Q_{eps_eff}(G^n) on the grid (transform, Lemma sums, combination, inverse transform);
  3. (a) rho, u, e advanced with the moments of Q^n (Delta xi = (2 pi / N)^d, collision frequency
         c = 1: the homogeneous equation d_t f = Q(f) that the rest of this project steps);
     (b) the temperature T^{n+1} (and the fugacity z^{n+1}) from rho^{n+1}, e^{n+1}: T = 2 e / d
         classically; for eps != 0 the equilibrium relations (mom02_qmaxwell) solved for z by
         Brent's method, on mu = ln z for Fermi-Dirac particles (Sec. 1.2);
     (c) w^{n+1} = sqrt(T^{n+1}) (quantum), sqrt(T^{n+1} + |u^{n+1}|^2 / d) (classical);
  4. the divergence term div((a xi - b) G^n), a = (w^{n+1} - w^n) / (dt w^n),
     b = (pi w^n / L)(u^{n+1} - u^n) / dt, by spectral differentiation: the modes of each flux
     component times i k_d (k_d in I_N; the k_d = -N/2 mode, which has no partner, gets 0);
  5. G^{n+1} = G^n + dt (-div + (pi w^n / L)^{-gamma} Q^n).

The Fermi-Dirac and Bose-Einstein integrals of order 1 and 2 (2-D) are closed forms: K_1 = ln(1 + z)
or -ln(1 - z), K_2 = -Li_2(-z) or Li_2(z), the dilogarithm taken from scipy (spence(1 - x) = Li_2(x)).
Those of order 3/2 and 5/2 (3-D) are their defining integrals (Sec. 1.2) taken by scipy's adaptive
quadrature.
"""
from __future__ import annotations

import math
import warnings

import numpy as np
from scipy import integrate, optimize, special

from . import Operator


def li2(x: float) -> float:
    """The dilogarithm Li_2(x) = sum_k x^k / k^2 (x <= 1): the series itself for |x| < 1/2 (where
    1 - x rounds away the argument of Spence's function), scipy's Spence function otherwise."""
    if abs(x) < 0.5:
        total, term, k = 0.0, x, 1
        while True:
            add = term / (k * k)
            total += add
            if abs(add) <= 1e-18 * abs(total):
                return total
            k += 1
            term *= x
    return float(special.spence(1.0 - x))


def k_nu(nu: int, z: float, eps: float) -> float:
    """K_nu(z) of Sec. 1.2 for nu = 1, 2: the Fermi-Dirac integral (eps < 0) or the Bose-Einstein
    integral (eps > 0, 0 < z < 1)."""
    if eps < 0:
        return math.log1p(z) if nu == 1 else -li2(-z)
    return -math.log1p(-z) if nu == 1 else li2(z)


def k_half(nu: float, mu: float, eps: float) -> float:
    """K_nu(e^mu) of Sec. 1.2 for nu = 3/2, 5/2: Gamma(nu)^{-1} int_0^inf x^{nu-1} / (e^{x-mu} + s) dx,
    s = +1 Fermi-Dirac (eps < 0), -1 Bose-Einstein (eps > 0, mu < 0).  Written in t = sqrt(x),
    2 t^{2nu-1} / (e^{t^2-mu} + s), split at t = sqrt(mu) (the Fermi step) when mu > 0 and cut where
    e^{t^2-mu} exceeds e^{60}."""
    fd = eps < 0

    def f(t):
        a = t * t - mu
        if a > 700.0:
            return 0.0
        return 2.0 * t ** (2.0 * nu - 1.0) / (math.exp(a) + 1.0 if fd else math.expm1(a))

    t0 = math.sqrt(max(mu, 0.0))
    t1 = math.sqrt(max(mu, 0.0) + 60.0)
    if t0 > 0.0:
        pts = [0.0, t0, t1]
    else:
        # Bose-Einstein near z = 1: below t ~ sqrt(-mu) the integrand drops from 2 t^{2nu-1} / t^2 to
        # 0, a layer that carries a relative pi sqrt(-mu) / K; breakpoints at sqrt(-mu) 10^k resolve it
        pts = [0.0]
        if not fd:
            c = max(math.sqrt(-mu), 1e-17)
            while c < 1.0:
                pts.append(c)
                c *= 10.0
        pts.append(t1)
    pieces = list(zip(pts[:-1], pts[1:]))
    total = 0.0
    with warnings.catch_warnings():
        # quad reports roundoff at the tolerance it is asked for; the pins bound the result (1e-14)
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        for a, b in pieces:
            v, _ = integrate.quad(f, a, b, epsabs=0.0, epsrel=1.2e-14, limit=500)
            total += v
    return total / special.gamma(nu)


# the ends of I_eq in 3-D (def_Ieq)
IEQ_FD_3D = 5.0 / 3.0 * math.sqrt(10.0 / math.pi)
IEQ_BE_3D = float(special.zeta(1.5)) ** 2.5 / float(special.zeta(2.5)) ** 1.5


def _temperature_3d(eps: float, rho: float, e: float):
    """3-D: nu = 3/2, x = |eps| rho (3 / (4 pi e))^{3/2} = K_{3/2}^{5/2} / K_{5/2}^{3/2} (eq_fugacity),
    compared in logarithms; Brent on mu = ln z (Fermi-Dirac) or on ln(-mu) (Bose-Einstein, so that
    z -> 1 stays resolved); T = (|eps| rho / K_{3/2})^{2/3} / (2 pi) (mom0_qmaxwell)."""
    x = abs(eps) * rho * (3.0 / (4.0 * math.pi * e)) ** 1.5
    lx = math.log(x) if x > 0.0 else -math.inf

    def g(mu):
        return 2.5 * math.log(k_half(1.5, mu, eps)) - 1.5 * math.log(k_half(2.5, mu, eps)) - lx

    if eps < 0:
        if not 0.0 < x < IEQ_FD_3D:
            raise ValueError("Fermi-Dirac moments outside I_eq (degenerate state)")
        if g(700.0) < 0.0:
            raise ValueError("the fugacity lies beyond ln z = 700")
        mu = optimize.brentq(g, -600.0, 700.0, xtol=1e-14, rtol=1e-15, maxiter=500)
    else:
        if not 0.0 < x < IEQ_BE_3D:
            raise ValueError("Bose-Einstein moments outside I_eq (condensed state)")
        lam = optimize.brentq(lambda l: g(-math.exp(l)), -690.0, math.log(600.0), xtol=1e-14, rtol=1e-15,
                              maxiter=500)
        mu = -math.exp(lam)
    T = (abs(eps) * rho / k_half(1.5, mu, eps)) ** (2.0 / 3.0) / (2.0 * math.pi)
    return T, math.exp(mu)


def temperature(d: int, eps: float, rho: float, e: float):
    """(T, z) from the mass and internal energy (Sec. 3.3 step 3(b); Sec. 1.2): classical T = 2e/d
    (z = None); quantum: x = |eps| rho (d / (4 pi e))^{d/2} must lie in I_eq (2-D: (0, 2) for
    Fermi-Dirac, (0, inf) for Bose-Einstein; 3-D: see _temperature_3d); in 2-D z solves
    x = K_1(z)^2 / K_2(z) (eq_fugacity with nu = 1) and T = (|eps| rho / K_1(z)) / (2 pi)
    (mom0_qmaxwell).  Raises ValueError outside I_eq."""
    if eps == 0.0:
        return 2.0 * e / d, None
    if d == 3:
        return _temperature_3d(eps, rho, e)
    x = abs(eps) * rho * (d / (4.0 * math.pi * e)) ** (d / 2.0)
    if eps < 0:
        if not 0.0 < x < 2.0:
            raise ValueError("Fermi-Dirac moments outside I_eq (degenerate state)")
        g = lambda mu: k_nu(1, math.exp(mu), eps) ** 2 / k_nu(2, math.exp(mu), eps) - x
        z = math.exp(optimize.brentq(g, -60.0, 60.0, xtol=1e-15, rtol=1e-15, maxiter=500))
    else:
        if not x > 0.0:
            raise ValueError("Bose-Einstein moments outside I_eq")
        g = lambda zz: k_nu(1, zz, eps) ** 2 / k_nu(2, zz, eps) - x
        z = optimize.brentq(g, 1e-300, 1.0 - 1e-16, xtol=1e-300, rtol=1e-15, maxiter=500)
    T = abs(eps) * rho / k_nu(1, z, eps) / (2.0 * math.pi)
    return T, z


def omega_of(d: int, eps: float, T: float, u) -> float:
    """The velocity scale of Sec. 3.3 step 3(c)."""
    if eps != 0.0:
        return math.sqrt(T)
    return math.sqrt(T + float(np.dot(u, u)) / d)


def xi_grid(d: int, N: int) -> np.ndarray:
    """xi_j = 2 pi j / N, j in I_N, as an (N,)*d + (d,) array."""
    j = np.arange(-N // 2, N // 2) * (2.0 * math.pi / N)
    return np.stack(np.meshgrid(*([j] * d), indexing="ij"), axis=-1)


def spectral_divergence(H: np.ndarray) -> np.ndarray:
    """sum_d d/dxi_d H_d on the periodic grid of [-pi, pi]^d: the modes of each component (the
    transform of Sec. 3.3 step 2(a), here by numpy's FFT with the I_N ordering) times i k_d, the
    k_d = -N/2 mode set to 0, transformed back; H has shape (N,)*d + (d,)."""
    d = H.shape[-1]
    N = H.shape[0]
    k = np.fft.fftfreq(N, 1.0 / N)          # 0, 1, ..., N/2 - 1, -N/2, ..., -1
    k[N // 2] = 0.0                        # the unpaired -N/2 mode
    out = np.zeros(H.shape[:-1])
    for c in range(d):
        Hc = np.fft.ifftshift(H[..., c])   # grid index j = -N/2 .. N/2-1 -> FFT order
        F = np.fft.fftn(Hc)
        shape = [1] * d
        shape[c] = N
        F = F * (1j * k.reshape(shape))
        out += np.fft.fftshift(np.fft.ifftn(F).real)
    return out


class RescaledRun:
    """The state of one rescaled solve (d = 2, or d = 3 classically): G on the xi grid, rho, u, e, w,
    and the operator (box pi, truncation R) whose eps is set to eps (pi w / L)^d before every
    evaluation; `op_kw` goes to the operator (3-D: M1, M2)."""

    def __init__(self, N: int, L: float, R: float, kernel: int, eps: float, G, rho: float, u, e: float, w: float,
                 d: int = 2, **op_kw):
        self.d, self.N, self.L, self.eps = int(d), int(N), float(L), float(eps)
        self.gamma = 1 if kernel == 1 else 0
        self.op = Operator(self.d, self.N, math.pi, R, kernel, 0.0, **op_kw)
        self.G = np.array(G, dtype=np.float64).reshape((self.N,) * self.d)
        self.rho, self.u, self.e, self.w = float(rho), np.array(u, dtype=np.float64), float(e), float(w)
        self.T, self.z = None, None
        self.xi = xi_grid(self.d, self.N)

    def scale(self) -> float:
        return math.pi * self.w / self.L

    def collision(self) -> np.ndarray:
        """Q_{eps (pi w / L)^d}(G) on the grid (the operator of the box [-pi, pi]^d)."""
        self.op.eps = self.eps * self.scale() ** self.d
        return self.op.eval_collision(self.G)

    def moments_update(self, Q: np.ndarray, dt: float):
        """Step 3(a): rho^{n+1}, u^{n+1}, e^{n+1} from the moments of Q^n."""
        d, N, s = self.d, self.N, self.scale()
        coef = (2.0 * math.pi / N) ** d * s ** (-self.gamma)
        S0 = float(Q.sum())
        S1 = np.array([float((self.xi[..., c] * Q).sum()) for c in range(d)])
        S2 = float((np.sum(self.xi ** 2, axis=-1) * Q).sum())
        rho1 = self.rho + dt * coef * S0
        rhou1 = self.rho * self.u + dt * coef * (S1 / s + self.u * S0)
        rhoe1 = self.rho * self.e + dt * 0.5 * coef * S2 / s ** 2
        return rho1, rhou1 / rho1, rhoe1 / rho1

    def advance(self, Q: np.ndarray, dt: float, w1: float, u1) -> np.ndarray:
        """Steps 4-5: G^{n+1} from G^n, Q^n and the new scale w^{n+1} and mean velocity u^{n+1}."""
        s = self.scale()
        a = (w1 - self.w) / (dt * self.w)
        b = s * (np.asarray(u1, dtype=np.float64) - self.u) / dt
        div = spectral_divergence((a * self.xi - b) * self.G[..., None])
        return self.G + dt * (-div + s ** (-self.gamma) * Q)

    def step(self, dt: float):
        """One forward Euler step of Sec. 3.3 (steps 2 to 5)."""
        Q = self.collision()
        rho1, u1, e1 = self.moments_update(Q, dt)
        T1, z1 = temperature(self.d, self.eps, rho1, e1)
        w1 = omega_of(self.d, self.eps, T1, u1)
        self.G = self.advance(Q, dt, w1, u1)
        self.rho, self.u, self.e, self.w, self.T, self.z = rho1, u1, e1, w1, T1, z1
        return self

    def rhs(self, G, Q, s: float, a: float, b) -> np.ndarray:
        """F(G) = -div((a xi - b) G) + s^{-gamma} Q: the right-hand side of the rescaled equation at
        scale s with dilation rate a = w'/w and drift b = (pi w / L) u'."""
        div = spectral_divergence((a * self.xi - np.asarray(b, dtype=np.float64)) * G[..., None])
        return -div + s ** (-self.gamma) * Q

    def step_rk2(self, dt: float):
        """One step of the SSP-RK2 (Heun) form of the procedure (reading of the RK2 variant the
        paper mentions for Sec. 3.3):
          predictor: the forward Euler step (G1, rho1, u1, e1, w1 from Q0 = Q(G0));
          moments:   Y^{n+1} = (Y^n + Y^(2)) / 2 for rho, rho u, rho e, Y^(2) the Euler moment update
                     from (rho1, u1, e1) with the moments of Q1 = Q(G1) at the scale of G1;
                     T, z, w^{n+1} from the averaged rho, e (steps 3(b), (c));
          G:         G^{n+1} = G0 + dt/2 [F(G0) + F(G1)], F at each stage's own scale, with the
                     midpoint rates a = ln(w^{n+1} / w^n) / dt and u' = (u^{n+1} - u^n) / dt."""
        G0, rho0, u0, e0, w0 = self.G.copy(), self.rho, self.u.copy(), self.e, self.w
        s0 = self.scale()
        Q0 = self.collision()
        rho1, u1, e1 = self.moments_update(Q0, dt)
        T1, _ = temperature(self.d, self.eps, rho1, e1)
        w1 = omega_of(self.d, self.eps, T1, u1)
        G1 = self.advance(Q0, dt, w1, u1)
        # the second stage, from the predictor
        self.G, self.rho, self.u, self.e, self.w = G1, rho1, u1, e1, w1
        s1 = self.scale()
        Q1 = self.collision()
        rho2, u2, e2 = self.moments_update(Q1, dt)
        rhoN = 0.5 * (rho0 + rho2)
        uN = 0.5 * (rho0 * u0 + rho2 * u2) / rhoN
        eN = 0.5 * (rho0 * e0 + rho2 * e2) / rhoN
        TN, zN = temperature(self.d, self.eps, rhoN, eN)
        wN = omega_of(self.d, self.eps, TN, uN)
        a = math.log(wN / w0) / dt
        du = (uN - u0) / dt
        self.G = G0 + 0.5 * dt * (self.rhs(G0, Q0, s0, a, s0 * du) + self.rhs(G1, Q1, s1, a, s1 * du))
        self.rho, self.u, self.e, self.w, self.T, self.z = rhoN, uN, eN, wN, TN, zN
        return self

    def f_grid(self):
        """(v, f): the velocities v_j = u + 2 L j / (N w) and f_j = (pi w / L)^d G_j."""
        s = self.scale()
        return self.u + self.xi / s, s ** self.d * self.G
