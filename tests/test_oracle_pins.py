"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test pins the oracle to something other than itself:
  * closed forms of the kernel modes beta(0,0), beta(k,0), beta(0,l) derived from
    their definition (Lemma of Sec. 2.3) -- pins phi, psi, C_Phi and the quadrature;
  * symmetries beta(+-a,+-b) that follow from the definition;
  * an independent brute-force quadrature of the truncated Carleman integral
    (Sec. 2.2) for band-limited G -- pins every per-term label, sign and constant
    of the Lemma's sums and of the combination Q1c - Q2c - alpha[Q1q+Q2q-Q3q-Q4q];
  * exact conservation of mass and spectral conservation of momentum/energy
    (eq. conservationQ);
  * the 2-D BKW exact solution for Maxwell molecules (literature) -- pins the
    classical scaling (T/pi)^{d+gamma} and C_Phi, and RK4 in time;
  * quantum Maxwellians (Sec. 1.2): Q ~ 0 with alpha = -eps and the printed
    fugacities and residual tables (tests/golden) -- pins the sign of eps;
  * the closed-form loss term of a Gaussian (hard spheres and Maxwell) -- pins
    gamma in the prefactor and beta(l,l);
  * closed-form moments of a Gaussian (Sec. 4 head).
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest
from scipy import special

import oracle as O
from paper_2110_13735_gb300 import inputs as I
from tests import equilibria as EQ
from tests.carleman import carleman_2d, carleman_3d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
R6 = 6.0
T6 = I.box_half_width(R6)
RXI = 2 * math.pi / (3 + math.sqrt(2))


def _op(d, N, eps=0.0, **kw):
    return O.Operator(d, N, T6, R6, 0 if d == 2 else 1, eps, **kw)


# --------------------------------------------------------------------------- beta
def test_beta_closed_forms_2d():
    """beta(0,0) = 4 pi R^2 Btilde; beta(k,0) = beta(0,k) = 4 pi R Btilde int_0^R J0(rho|k|) drho
    (delta(z.y) restricted to B_R x B_R; Btilde = 2 C_Phi for 2-D Maxwell molecules)."""
    op = _op(2, 8, M=64)
    Bt = 2 * op.c_phi
    assert op.beta_at((0, 0), (0, 0)) == pytest.approx(4 * math.pi * RXI ** 2 * Bt, rel=1e-13)
    for k in [(1, 0), (2, 3), (-4, 1), (3, -3), (-8, 7)]:
        q = math.hypot(*k)
        intj0 = special.itj0y0(RXI * q)[0] / q
        exact = 4 * math.pi * RXI * Bt * intj0
        assert op.beta_at(k, (0, 0)) == pytest.approx(exact, rel=1e-11, abs=1e-13)
        assert op.beta_at((0, 0), k) == pytest.approx(exact, rel=1e-11, abs=1e-13)


def test_beta_hard_spheres_2d_closed_form_and_order():
    """2-D hard spheres (reading r5): beta(0,0) = 2 C_Phi pi int int_{[-R,R]^2} sqrt(x^2+y^2)
    = 2 C_Phi pi (4 R^3 / 3)(sqrt 2 + asinh 1).  The tensor Gauss-Legendre rule meets it at
    third order (the integrand has a conical point at the origin): the error falls ~8x per
    doubling of Q and is below 1e-6 at Q = 96."""
    exact = None
    errs = []
    for Q in (24, 48, 96):
        op = O.Operator(2, 4, T6, R6, 1, 0.0, M=16, Q=Q)
        exact = 2 * op.c_phi * math.pi * (4 * RXI ** 3 / 3) * (math.sqrt(2) + math.asinh(1))
        errs.append(abs(op.beta_at((0, 0), (0, 0)) / exact - 1))
    assert errs[2] < 1e-6
    assert 5 < errs[0] / errs[1] < 12 and 5 < errs[1] / errs[2] < 12


def test_beta_closed_forms_3d():
    """3-D hard spheres: beta(0,0) = 2 pi^2 R^4 Btilde, beta(k,0) = beta(0,k) =
    4 pi^2 R^2 Btilde (1-cos R|k|)/|k|^2 (Btilde = 4 C_Phi)."""
    op = _op(3, 4, M1=24, M2=24)
    Bt = 4 * op.c_phi
    assert op.beta_at((0, 0, 0), (0, 0, 0)) == pytest.approx(2 * math.pi ** 2 * RXI ** 4 * Bt, rel=1e-12)
    for k in [(1, 0, 0), (1, 2, -3), (-4, 3, 2), (3, 3, 3)]:
        q = math.sqrt(sum(x * x for x in k))
        exact = 4 * math.pi ** 2 * RXI ** 2 * Bt * (1 - math.cos(RXI * q)) / q ** 2
        assert op.beta_at(k, (0, 0, 0)) == pytest.approx(exact, rel=1e-11)
        assert op.beta_at((0, 0, 0), k) == pytest.approx(exact, rel=1e-11)


def test_printed_3d_theta_rule_is_second_order():
    """Reading r3: with the printed sin(theta_p)-weighted rectangle rule the error of
    beta(k,0) falls by ~4x per doubling of M1 (second order), while the Gauss rule is exact."""
    k = (3, 1, 2)
    q = math.sqrt(14.0)
    errs = []
    for M1 in (8, 16, 32):
        op = O.Operator(3, 4, T6, R6, 1, 0.0, M1=M1, M2=M1, quad3d=1)
        exact = 4 * math.pi ** 2 * RXI ** 2 * 4 * op.c_phi * (1 - math.cos(RXI * q)) / q ** 2
        errs.append(abs(op.beta_at(k, (0, 0, 0)) - exact) / exact)
    assert errs[0] > 1e-2
    assert 3.0 < errs[0] / errs[1] < 5.5 and 3.0 < errs[1] / errs[2] < 5.5


@pytest.mark.parametrize("d,N,kw", [(2, 6, dict(M=12)), (3, 4, dict(M1=8, M2=8))])
def test_beta_symmetries(d, N, kw):
    """beta(a,b) = beta(-a,b) = beta(a,-b) (z -> -z, y -> -y in the definition); for a
    constant Btilde beta(a,b) = beta(b,a) (exactly in 2-D with even M, to quadrature
    accuracy in 3-D)."""
    op = _op(d, N, **kw)
    E = 2 * N
    beta = op.beta().reshape((E,) * (2 * d))
    # index of -a is E - (a+N) - N ... only for a in [-N+1, N-1]
    sl = tuple([slice(1, E)] * d)
    inner = beta[sl + sl]
    flip_a = inner[tuple([slice(None, None, -1)] * d) + (slice(None),) * d]
    flip_b = inner[(slice(None),) * d + tuple([slice(None, None, -1)] * d)]
    scale = np.abs(inner).max()
    assert np.abs(inner - flip_a).max() <= 1e-13 * scale
    assert np.abs(inner - flip_b).max() <= 1e-13 * scale
    perm = tuple(range(d, 2 * d)) + tuple(range(d))
    sym_err = np.abs(inner - np.transpose(inner, perm)).max() / scale
    assert sym_err <= (1e-13 if d == 2 else 1e-2)


# --------------------------------------------------------------------------- DFT
def test_dft_conventions():
    """G^_k = N^-d sum_j G_j e^{-2 i pi k.j/N} recovers the coefficient of a pure mode;
    the inverse returns the real part of sum_n Q^_n e^{2 i pi n.j/N}."""
    N = 8
    op = _op(2, N)
    j = np.arange(-N // 2, N // 2)
    J0, J1 = np.meshgrid(j, j, indexing="ij")
    k0 = (2, -3)
    f = np.cos(2 * np.pi * (k0[0] * J0 + k0[1] * J1) / N)
    Gh = op.dft(f)
    ref = np.zeros((N, N), complex)
    ref[k0[0] + N // 2, k0[1] + N // 2] += 0.5
    ref[-k0[0] + N // 2, -k0[1] + N // 2] += 0.5
    assert np.abs(Gh - ref).max() < 1e-14
    rng = np.random.Generator(np.random.PCG64(1))
    g = rng.standard_normal((N, N))
    assert np.abs(op.idft_real(op.dft(g)) - g).max() < 1e-13


# --------------------------------------------------------------------------- brute force
def _random_modes(d, N, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = np.arange(-N // 2, N // 2)
    K = np.stack(np.meshgrid(*([ks] * d), indexing="ij"), -1)
    decay = np.exp(-0.15 * np.sum(K * K, -1))
    return (rng.standard_normal(K.shape[:-1]) + 1j * rng.standard_normal(K.shape[:-1])) * decay * 0.3


@pytest.mark.parametrize("eps", [0.0, 1.0, -1.0, 2.5])
def test_brute_force_carleman_2d(eps):
    """Lemma sums (unprojected modes) vs direct quadrature of Q^R_alpha(G)(xi), 2-D N=8."""
    N = 8
    op = _op(2, N, eps=eps, M=64)
    Gh = _random_modes(2, N, 11 + int(10 * eps))
    lo, cnt = -3 * N // 2, 3 * N - 2
    Qh = op.collision_modes(Gh, lo, cnt)[0]
    nn = np.arange(lo, lo + cnt)
    NN = np.stack(np.meshgrid(nn, nn, indexing="ij"), -1).reshape(-1, 2)
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(3):
        xi = rng.uniform(-np.pi, np.pi, 2)
        lemma = np.sum(Qh.reshape(-1) * np.exp(1j * (NN @ xi)))
        bf = carleman_2d(Gh, N, RXI, 2 * op.c_phi, -eps, xi)
        assert abs(lemma - bf) <= 1e-11 * max(1.0, abs(bf))


@pytest.mark.parametrize("eps", [0.0, 1.0, -1.0])
def test_brute_force_carleman_2d_hard_spheres(eps):
    """2-D hard spheres (reading r5), Btilde = 2 C_Phi sqrt(|x|^2+|y|^2): Lemma sums vs the
    direct Carleman quadrature with the same radial rule.  Pins the (theta, rho') separable
    form of the kernel modes, its weights and the square root."""
    N = 8
    op = O.Operator(2, N, T6, R6, 1, eps, M=64, Q=48)
    Gh = _random_modes(2, N, 31 + int(10 * eps))
    lo, cnt = -3 * N // 2, 3 * N - 2
    Qh = op.collision_modes(Gh, lo, cnt)[0]
    nn = np.arange(lo, lo + cnt)
    NN = np.stack(np.meshgrid(nn, nn, indexing="ij"), -1).reshape(-1, 2)
    rng = np.random.Generator(np.random.PCG64(5))
    bt = lambda x, y: 2 * op.c_phi * np.sqrt(x * x + y * y)
    for _ in range(2):
        xi = rng.uniform(-np.pi, np.pi, 2)
        lemma = np.sum(Qh.reshape(-1) * np.exp(1j * (NN @ xi)))
        bf = carleman_2d(Gh, N, RXI, bt, -eps, xi, n_rho=48)
        assert abs(lemma - bf) <= 1e-11 * max(1.0, abs(bf))


@pytest.mark.parametrize("eps", [1.0, -1.0])
def test_brute_force_carleman_3d(eps):
    """Same pin in 3-D (hard spheres, N=4): pins psi (reading r2) and the 3-D beta."""
    N = 4
    op = _op(3, N, eps=eps, M1=24, M2=48)
    Gh = _random_modes(3, N, 21 + int(eps))
    lo, cnt = -3 * N // 2, 3 * N - 2
    Qh = op.collision_modes(Gh, lo, cnt)[0]
    nn = np.arange(lo, lo + cnt)
    NN = np.stack(np.meshgrid(nn, nn, nn, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.Generator(np.random.PCG64(4))
    xi = rng.uniform(-np.pi, np.pi, 3)
    lemma = np.sum(Qh.reshape(-1) * np.exp(1j * (NN @ xi)))
    bf = carleman_3d(Gh, N, RXI, 4 * op.c_phi, -eps, xi)
    assert abs(lemma - bf) <= 1e-11 * max(1.0, abs(bf))


# --------------------------------------------------------------------------- conservation
@pytest.mark.parametrize("d,N,eps", [(2, 16, -1.0), (2, 16, 1.0), (2, 16, 0.0), (3, 8, -1.0), (3, 8, 1.0)])
def test_mass_exact(d, N, eps):
    """sum_j Q_j = N^d Re Q^_0 = 0 up to rounding (the four cubic weights coincide when
    k+l+m = 0 and beta is even; the quadratic part cancels through beta(k,-k) = beta(k,k))."""
    op = _op(d, N, eps=eps, M=2 * N) if d == 2 else _op(d, N, eps=eps, M1=8, M2=8)
    rng = np.random.Generator(np.random.PCG64(7))
    T = op.T
    f = I.two_gaussians(d, N, T, 1.0, (1.5,) + (0.5,) * (d - 1), 0.8) * (1 + 0.1 * rng.uniform(size=(N,) * d))
    Q, gain, loss, cub = op.eval_collision(f, parts=True)
    assert abs(Q.sum()) <= 1e-13 * np.abs(gain).sum()


def _mom_energy_defect(N, eps):
    op = _op(2, N, eps=eps, M=N)
    f = I.config0_f0(N)
    Q, gain, _, _ = op.eval_collision(f, parts=True)
    v = op.velocities()
    scale = np.sum(np.abs(gain) * np.sum(v * v, -1))
    mom = np.abs(np.tensordot(Q, v, axes=([0, 1], [0, 1]))).max()
    en = abs(np.sum(Q * np.sum(v * v, -1)))
    return max(mom, en) / scale


def test_momentum_energy_spectral():
    """int Q v dv and int Q |v|^2 dv vanish to spectral accuracy: the defect relative to the
    gain term falls by more than 10x from N=16 to N=32 (eps=-1) and by more than 5x from N=32 to N=40
    (eps=0)."""
    r16, r32 = _mom_energy_defect(16, -1.0), _mom_energy_defect(32, -1.0)
    assert r32 < 1e-4 and r32 < 0.1 * r16
    assert _mom_energy_defect(40, 0.0) < 0.2 * _mom_energy_defect(32, 0.0)


# --------------------------------------------------------------------------- BKW
def test_bkw_operator_convergence():
    """Q(f_BKW(1)) vs d/dt f_BKW(1) (2-D Maxwell, B = 1/(2 pi), eps = 0): relative max error
    below 5e-2 at N=32 and 2e-3 at N=48 (spectral convergence of the classical part)."""
    for N, tol in ((32, 5e-2), (48, 2e-3)):
        op = _op(2, N, eps=0.0, M=N)
        v = op.velocities()
        Q = op.eval_collision(I.bkw_2d(1.0, v))
        ref = I.bkw_2d_dt(1.0, v)
        assert np.abs(Q - ref).max() / np.abs(ref).max() < tol


def test_rk4_bkw_time_order():
    """RK4 on the BKW datum: the time error against a fine-step run shrinks ~16x per halving
    of dt (fourth order), and SSP-RK2 ~4x (second order)."""
    N = 16
    op = _op(2, N, eps=0.0, M=N)
    f0 = I.bkw_2d(1.0, op.velocities())
    ref = op.step(f0, 0.0125, 32, 0)
    e1 = np.abs(op.step(f0, 0.2, 2, 0) - ref).max()
    e2 = np.abs(op.step(f0, 0.1, 4, 0) - ref).max()
    assert 12.0 < e1 / e2 < 20.0
    s1 = np.abs(op.step(f0, 0.1, 4, 1) - ref).max()
    s2 = np.abs(op.step(f0, 0.05, 8, 1) - ref).max()
    assert 3.0 < s1 / s2 < 5.0


def test_rk4_follows_bkw_in_time():
    """Integrating the BKW datum from t=1 to t=2 at N=48 stays within 2e-3 of the exact solution."""
    N = 48
    op = _op(2, N, eps=0.0, M=N)
    v = op.velocities()
    f = op.step(I.bkw_2d(1.0, v), 0.1, 10, 0)
    ref = I.bkw_2d(2.0, v)
    assert np.abs(f - ref).max() / np.abs(ref).max() < 2e-3


# --------------------------------------------------------------------------- equilibria
def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_printed_fugacities_reproduce_mass():
    """Every fugacity printed in the Sec. 4.1 captions reproduces rho with T = sigma, hbar = 3."""
    for d, stat, rho, sig, z, *_ in _golden("fugacities.txt"):
        d, rho, sig, z = int(d), float(rho), float(sig), float(z)
        m = EQ.mass(d, stat, z, sig, 3.0 ** d)
        assert m == pytest.approx(rho, rel=2e-4), (d, stat, rho, sig, z, m)
        zs = EQ.fugacity(d, stat, rho, sig, 3.0 ** d)
        assert zs == pytest.approx(z, rel=2e-4)


@pytest.mark.parametrize("stat,L,sig", [("FD", 6.0, 1.0), ("FD", 4.0, 0.5), ("BE", 6.0, 1.0)])
def test_quantum_maxwellian_residual(stat, L, sig):
    """Q_eps(M_q) ~ 0 for the quantum Maxwellian with eps = -alpha (alpha = +-hbar^2, hbar=3):
    the residual is far below the gain term, decays from N=16 to 32, and is no larger than the
    paper's printed residual (the direct sum has no extra quadrature/aliasing error).  With the
    opposite sign of eps the residual is of the order of the gain term."""
    d, hbar = 2, 3.0
    alpha = hbar ** d if stat == "FD" else -hbar ** d
    z = EQ.fugacity(d, stat, 1.0, sig, abs(alpha))
    Rv = 2 * L / (3 + math.sqrt(2))
    printed = {int(r[3]): float(r[4]) for r in _golden("residuals_2d.txt")
               if r[0] == stat and float(r[1]) == L and float(r[2]) == sig}
    res = {}
    for N in (16, 32):
        op = O.Operator(2, N, L, Rv, 0, -alpha, M=N)
        f = EQ.quantum_maxwellian(op.velocities(), stat, z, sig, abs(alpha))
        Q, gain, _, _ = op.eval_collision(f, parts=True)
        res[N] = np.abs(Q).max()
        assert res[N] <= printed[N]
        assert res[N] < (1e-1 if N == 16 else 1e-2) * np.abs(gain).max()
        if N == (16 if stat == "FD" else 32):
            wrong = O.Operator(2, N, L, Rv, 0, alpha, M=N).eval_collision(f)
            assert np.abs(wrong).max() > 10.0 * res[N]
    assert res[32] < res[16]


# --------------------------------------------------------------------------- loss term scale
def test_loss_term_gaussian_closed_form():
    """Q^-(f)(0) = f(0) |S^{d-1}| C_Phi int |v_*|^gamma f(v_*) dv_*: for a Gaussian of mass rho
    and temperature T this is f(0) 2 pi C_Phi rho (2-D Maxwell) and f(0) 4 pi C_Phi rho
    sqrt(8T/pi) (3-D hard spheres).  Pins (T/pi)^{d+gamma}, C_Phi and beta(l,l).  The
    tolerance 1e-3 covers the spectral error of a unit-temperature Gaussian on these grids
    (Nyquist pi/h ~ 3.8 in 2-D: e^{-(pi/h)^2/2} ~ 7e-4); a wrong gamma or C_Phi is off by
    factors of T/pi ~ 4 or 2 pi."""
    rho, temp = 1.0, 1.0
    op2 = _op(2, 32, M=32)
    f2 = I.gaussian(2, 32, T6, rho, temp)
    _, _, loss2, _ = op2.eval_collision(f2, parts=True)
    exact2 = f2[16, 16] * 2 * math.pi * op2.c_phi * rho
    assert loss2[16, 16] == pytest.approx(exact2, rel=1e-3)
    # 3-D N=16: a wider Gaussian (temperature 3) balances the grid's spectral error against
    # the mass outside the truncation ball (both ~e^{-5.7} here), hence rel=2e-2.
    op3 = _op(3, 16, M1=12, M2=12)
    temp3 = 3.0
    f3 = I.gaussian(3, 16, T6, rho, temp3)
    _, _, loss3, _ = op3.eval_collision(f3, parts=True)
    exact3 = f3[8, 8, 8] * 4 * math.pi * op3.c_phi * rho * math.sqrt(8 * temp3 / math.pi)
    assert loss3[8, 8, 8] == pytest.approx(exact3, rel=2e-2)


def test_loss_term_gaussian_closed_form_2d_hard_spheres():
    """2-D hard spheres: Q^-(f)(0) = f(0) 2 pi C_Phi rho sqrt(pi T / 2) (the mean speed of a 2-D
    Gaussian).  Pins gamma = 1 in (T/pi)^{d+gamma} for d = 2 and the hard-sphere beta(l,l).  The
    tolerance 2e-2 covers the slower spectral convergence of the |v - v_*| weight on N = 16 (a
    wrong gamma is off by T/pi ~ 4)."""
    N, temp = 16, 3.0
    op = O.Operator(2, N, T6, R6, 1, 0.0, M=32)
    f = I.gaussian(2, N, T6, 1.0, temp)
    _, _, loss, _ = op.eval_collision(f, parts=True)
    exact = f[N // 2, N // 2] * 2 * math.pi * op.c_phi * math.sqrt(math.pi * temp / 2)
    assert loss[N // 2, N // 2] == pytest.approx(exact, rel=2e-2)


def test_hard_spheres_2d_mass_and_fermi_dirac_residual():
    """The hard-sphere operator conserves mass to rounding, and a Fermi-Dirac equilibrium
    (alpha = hbar^2, hbar = 3) is a near-zero of it with the right sign of eps only."""
    d, hbar, L, sig = 2, 3.0, 6.0, 1.0
    alpha = hbar ** d
    z = EQ.fugacity(d, "FD", 1.0, sig, alpha)
    Rv = 2 * L / (3 + math.sqrt(2))
    op = O.Operator(2, 16, L, Rv, 1, -alpha, M=16)
    f = EQ.quantum_maxwellian(op.velocities(), "FD", z, sig, alpha)
    Q, gain, _, _ = op.eval_collision(f, parts=True)
    assert abs(Q.sum()) <= 1e-13 * np.abs(gain).sum()
    res = np.abs(Q).max()
    assert res < 1e-1 * np.abs(gain).max()
    wrong = O.Operator(2, 16, L, Rv, 1, alpha, M=16).eval_collision(f)
    assert np.abs(wrong).max() > 10.0 * res


# --------------------------------------------------------------------------- moments
def test_moments_gaussian():
    """rho, u and e of a shifted Gaussian on the grid equal rho0, u0 and d T/2 to the spectral
    accuracy of the grid sum (~exp(-2 pi^2 T/h^2) ~ 1e-10 here)."""
    N = 32
    op = _op(2, N, eps=-1.0)
    u0 = np.array([0.7, -0.4])
    f = I.gaussian(2, N, T6, 2.0, 0.8, u=u0)
    m = op.moments(f)
    assert m[0] == pytest.approx(2.0, rel=1e-8)
    assert m[1:3] / m[0] == pytest.approx(u0, rel=1e-8)
    assert m[3] == pytest.approx(0.8, rel=1e-8)
    assert m[6] == pytest.approx(f.max(), rel=0)
