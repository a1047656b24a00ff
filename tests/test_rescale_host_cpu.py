"""The library's own temperature and fugacity solve of the velocity-rescaling step (include/bn.h:
bn_equilibrium_temperature; its dilogarithm from the series with Euler's reflection, Landen's identity
and the inversion formula, and its own Brent iteration), on the CPU, against the oracle's solve
(oracle/rescaling.py: scipy's Spence function and brentq) and against quantum Maxwellian moments
from quadrature (tests/equilibria.py): from nearly classical to strongly degenerate fermions
(z = e^30) and bosons close to z = 1."""
from __future__ import annotations

import math
import os
import sys

import numpy as np
import pytest

from oracle import rescaling as RS
from paper_2110_13735_gb300 import bn

sys.path.insert(0, os.path.dirname(__file__))
import equilibria as EQ  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    try:
        return bn.load()
    except RuntimeError as e:
        pytest.skip(str(e))


def _moments(stat, eps, T, z):
    rho = EQ.mass(2, stat, z, T, abs(eps))
    K1 = EQ.fd_integral(1.0, z) if stat == "FD" else EQ.be_integral(1.0, z)
    K2 = EQ.fd_integral(2.0, z) if stat == "FD" else EQ.be_integral(2.0, z)
    return rho, T * K2 / K1


@pytest.mark.parametrize("stat,eps", [("FD", -9.0), ("FD", -1.0), ("BE", 9.0), ("BE", 1.0)])
@pytest.mark.parametrize("T,z", [(1.0, 1e-6), (0.5, 0.3), (2.0, 0.95), (0.7, 5.0), (0.2, math.exp(30.0)),
                                 (1.3, 0.999999)])
def test_temperature_against_quadrature_and_the_oracle(lib, stat, eps, T, z):
    if stat == "BE" and z >= 1.0:
        pytest.skip("Bose-Einstein fugacity < 1")
    rho, e = _moments(stat, eps, T, z)
    Tl, zl = bn.equilibrium_temperature(2, eps, rho, e)
    To, zo = RS.temperature(2, eps, rho, e)
    assert Tl == pytest.approx(T, rel=1e-10) and zl == pytest.approx(z, rel=1e-9)
    assert Tl == pytest.approx(To, rel=1e-12) and zl == pytest.approx(zo, rel=1e-11)


def test_classical_and_errors(lib):
    assert bn.equilibrium_temperature(2, 0.0, 1.3, 0.7) == (0.7, 0.0)
    assert bn.equilibrium_temperature(3, 0.0, 1.3, 0.6)[0] == pytest.approx(0.4)
    with pytest.raises(bn.BNError) as ei:          # 2-D Fermi-Dirac outside I_eq
        bn.equilibrium_temperature(2, -9.0, 1.0, 9.0 / (2 * math.pi * 2.5))
    assert ei.value.status == -7
    for eps, xmax in ((-1.0, RS.IEQ_FD_3D), (1.0, RS.IEQ_BE_3D)):   # 3-D outside I_eq
        e = 0.75 * (1.0 / (1.001 * xmax)) ** (2.0 / 3.0) / math.pi       # x = 1.001 xmax
        with pytest.raises(bn.BNError) as ei:
            bn.equilibrium_temperature(3, eps, 1.0, e)
        assert ei.value.status == -7
        e_in = 0.75 * (1.0 / (0.999 * xmax)) ** (2.0 / 3.0) / math.pi    # x = 0.999 xmax: solvable
        Tl, zl = bn.equilibrium_temperature(3, eps, 1.0, e_in)
        To, zo = RS.temperature(3, eps, 1.0, e_in)
        assert Tl == pytest.approx(To, rel=1e-10) and zl == pytest.approx(zo, rel=1e-8)
    with pytest.raises(bn.BNError):
        bn.equilibrium_temperature(2, 1.0, -1.0, 1.0)
    # the oracle agrees on the degenerate boundary
    with pytest.raises(ValueError):
        RS.temperature(2, -9.0, 1.0, 9.0 / (2 * math.pi * 2.5))
    # 2-D Bose-Einstein: x = K_1^2 / K_2 -> infinity as z -> 1, but with z in FP64 (z <= 1 - 1e-16) x
    # reaches only ~6 ln(1e16)^2 / pi^2 = 824; beyond that neither solve has a root in its bracket
    x_ok, x_far = 500.0, 5000.0
    for x, solvable in ((x_ok, True), (x_far, False)):
        rho, e = 1.0, 9.0 * 1.0 / (2 * math.pi * x)
        if solvable:
            T, z = bn.equilibrium_temperature(2, 9.0, rho, e)
            assert z == pytest.approx(RS.temperature(2, 9.0, rho, e)[1], rel=1e-12) and 1 - z < 1e-10
        else:
            with pytest.raises(bn.BNError):
                bn.equilibrium_temperature(2, 9.0, rho, e)
            with pytest.raises(ValueError):
                RS.temperature(2, 9.0, rho, e)


@pytest.mark.parametrize("stat,eps", [("FD", -9.0), ("FD", -1.0), ("BE", 9.0), ("BE", 1.0)])
@pytest.mark.parametrize("T,z", [(1.0, 1e-6), (0.5, 0.3), (2.0, 0.95), (0.7, 5.0), (0.3, math.exp(12.0)),
                                 (1.3, 1 - 1e-6)])
def test_temperature_3d_against_quadrature_and_the_oracle(lib, stat, eps, T, z):
    if stat == "BE" and z >= 1.0:
        pytest.skip("Bose-Einstein fugacity < 1")
    rho = EQ.mass(3, stat, z, T, abs(eps))
    K32 = EQ.fd_integral(1.5, z) if stat == "FD" else EQ.be_integral(1.5, z)
    K52 = EQ.fd_integral(2.5, z) if stat == "FD" else EQ.be_integral(2.5, z)
    e = 1.5 * T * K52 / K32
    Tl, zl = bn.equilibrium_temperature(3, eps, rho, e)
    To, zo = RS.temperature(3, eps, rho, e)
    assert Tl == pytest.approx(T, rel=1e-10) and zl == pytest.approx(z, rel=1e-8)
    # the degenerate end is ill-conditioned (d ln z / d ln x ~ mu^3): 1e-12 up to mu = 12
    assert Tl == pytest.approx(To, rel=1e-12) and zl == pytest.approx(zo, rel=1e-11)


@pytest.mark.parametrize("eps", [9.0, 1.0])
@pytest.mark.parametrize("T,one_minus_z", [(0.8, 1e-10), (1.5, 1e-14)])
def test_temperature_3d_bosons_near_condensation(lib, eps, T, one_minus_z):
    """3-D bosons with 1 - z down to 1e-14: the moments from mpmath's polylogarithm (the plain
    quadrature of tests/equilibria.py misses the x^{-1/2} layer of B_{3/2} there); both solves give
    back T, and z to the resolution of a double next to 1."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    z = 1 - mpmath.mpf(one_minus_z)
    K32, K52 = mpmath.polylog(1.5, z), mpmath.polylog(2.5, z)
    rho = float((2 * mpmath.pi * T) ** 1.5 * K32 / abs(eps))
    e = float(1.5 * T * K52 / K32)
    Tl, zl = bn.equilibrium_temperature(3, eps, rho, e)
    To, zo = RS.temperature(3, eps, rho, e)
    assert Tl == pytest.approx(T, rel=1e-12) and To == pytest.approx(T, rel=1e-12)
    assert abs(zl - float(z)) <= 4e-16 and abs(zo - float(z)) <= 4e-16


def test_printed_fugacities_through_both_temperature_solves(lib):
    """The fugacities printed in the Sec. 4.1 captions (tests/golden/fugacities.txt; hbar = 3, T =
    sigma, 2-D and 3-D, Fermi-Dirac and Bose-Einstein): with the paper's rho and the internal energy
    e = (d/2) sigma K_{d/2+1}(z) / K_{d/2}(z) of the printed z (mom2_qmaxwell), the oracle's and the
    library's solves give back T = sigma and the printed z to its printed digits."""
    path = os.path.join(os.path.dirname(__file__), "golden", "fugacities.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 10
    for d, stat, rho, sig, z, *_ in rows:
        d, rho, sig, z = int(d), float(rho), float(sig), float(z)
        eps = -(3.0 ** d) if stat == "FD" else 3.0 ** d
        K = EQ.fd_integral if stat == "FD" else EQ.be_integral
        e = 0.5 * d * sig * K(0.5 * d + 1.0, z) / K(0.5 * d, z)
        for T, zz in (RS.temperature(d, eps, rho, e), bn.equilibrium_temperature(d, eps, rho, e)):
            assert T == pytest.approx(sig, rel=5e-4), (d, stat, rho, sig)
            assert zz == pytest.approx(z, rel=5e-4), (d, stat, rho, sig)
