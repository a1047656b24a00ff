"""Pins of the Appendix's transform evaluation of Q_{1,q} (oracle/appendix.py; Mouton & Rey,
Appendix A), on the CPU.

The Appendix's route (FFTs per node p and grid point j) is checked against computations that share
none of its steps:
* the Lemma's cubic sum (Sec. 2.3) by brute force over all (k, l) with every index reduced modulo
  N, beta read from the C oracle's full kernel-mode table (eq. betadD) at the reduced arguments;
* the C oracle's CIRCULAR cubic bracket Q1q + Q2q - Q3q - Q4q, with the other three terms by brute
  force;
* for modes supported in a small central box, where no index sum leaves I_N, the C oracle's LINEAR
  bracket (the Lemma itself);
* single modes G^ = delta_{k0}, whose sum has one term: beta(2k0, 2k0) at n = 3k0 (reduced).
A slip in the transform signs, the N^{-d} normalisations, the FFT ordering, the restriction of
the alpha tables to I_N or the exponent (k + l - n) of step 3 fails the first of these.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

import oracle as O
from oracle import appendix as AP

S_TRUNC = 2.0 * math.pi / (3.0 + math.sqrt(2.0))


def _wrap(x, N):
    return (x + N // 2) % N - N // 2


def _modes(d, N):
    return np.array(list(itertools.product(range(-N // 2, N // 2), repeat=d)), dtype=np.int64)


def _flat(a, N, E, off):
    f = np.zeros(a.shape[:-1], dtype=np.int64)
    for i in range(a.shape[-1]):
        f = f * E + (a[..., i] + off)
    return f


def _brute_terms(op, Ghat):
    """Per output n: (Q1q, Q2q - Q3q - Q4q) by brute force, CIRCULAR indices, beta from the table."""
    d, N = op.d, op.N
    B = op.beta()
    G = np.asarray(Ghat).reshape(-1)
    K = _modes(d, N)
    KK, LL = K[:, None, :], K[None, :, :]
    ik, il = _flat(KK, N, N, N // 2), _flat(LL, N, N, N // 2)
    ext = lambda a: _flat(a, N, 2 * N, N)                              # noqa: E731
    q1 = np.zeros(len(K), dtype=np.complex128)
    rest = np.zeros(len(K), dtype=np.complex128)
    for t, n in enumerate(K):
        M = _wrap(n - KK - LL, N)
        kpm, lpm = _wrap(KK + M, N), _wrap(LL + M, N)
        g3 = G[ik] * G[il] * G[_flat(M, N, N, N // 2)]
        q1[t] = (B[ext(kpm), ext(lpm)] * g3).sum()
        lp = np.broadcast_to(LL, M.shape)
        w = B[ext(lp), ext(M)] - B[ext(lpm), ext(lp)] - B[ext(lp), ext(lpm)]
        rest[t] = (w * g3).sum()
    shape = (N,) * d
    return q1.reshape(shape), rest.reshape(shape)


def _appendix(op, Ghat):
    al, ap = op.alpha_tables()
    return AP.q1q_appendix(Ghat, AP.alpha_on_IN(al, op.d, op.N), AP.alpha_on_IN(ap, op.d, op.N))


def _rand_modes(rng, d, N, support=None):
    shape = (N,) * d
    G = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if support is not None:
        k = np.arange(-N // 2, N // 2)
        mask = np.ones(shape, dtype=bool)
        for ax in range(d):
            sh = [1] * d
            sh[ax] = N
            mask &= (np.abs(k) <= support).reshape(sh)
        G = np.where(mask, G, 0.0)
    return G


CASES = [(2, 8, 0), (2, 6, 0), (2, 6, 1), (3, 4, 1), (3, 6, 1)]


@pytest.mark.parametrize("d,N,kernel", CASES)
def test_appendix_equals_the_circular_lemma_sum(d, N, kernel):
    rng = np.random.default_rng(1000 + 10 * d + N + kernel)
    kw = dict(Q=N + 2) if (d == 2 and kernel == 1) else {}
    op = O.Operator(d, N, math.pi, S_TRUNC, kernel, 1.0, wrap=1, **kw)
    G = _rand_modes(rng, d, N)
    fast = _appendix(op, G)
    q1, rest = _brute_terms(op, G)
    scale = np.abs(q1).max()
    assert np.abs(fast - q1).max() <= 1e-12 * scale
    # the C oracle's CIRCULAR cubic bracket, the other three terms added by brute force
    cubic = op.collision_modes(G)[3]
    assert np.abs(fast + rest - cubic).max() <= 1e-12 * np.abs(cubic).max()


@pytest.mark.parametrize("d,N,support", [(2, 12, 1), (3, 8, 1)])
def test_appendix_equals_the_linear_lemma_when_nothing_wraps(d, N, support):
    """Modes in |k_i| <= support with 3 support < N/2: every n, k+m, l+m stays in I_N, so the
    transform route gives the Lemma's (LINEAR) sum."""
    rng = np.random.default_rng(77 + N)
    kernel = 0 if d == 2 else 1
    lin = O.Operator(d, N, math.pi, S_TRUNC, kernel, 1.0, wrap=0)
    G = _rand_modes(rng, d, N, support=support)
    fast = _appendix(lin, G)
    q1, rest = _brute_terms(lin, G)
    cubic = lin.collision_modes(G)[3]
    assert np.abs(fast + rest - cubic).max() <= 1e-12 * np.abs(cubic).max()
    assert np.abs(fast - q1).max() <= 1e-12 * np.abs(q1).max()


@pytest.mark.parametrize("k0", [(0, 0), (1, -2), (3, 1), (-4, 2), (2, 3)])
def test_single_mode(k0):
    """G^ = delta_{k0}: the only triple is k = l = m = k0, so Q1q = beta(2k0, 2k0) at n = 3k0, all
    reduced into I_N (N = 8; k0 = (3, 1) and (2, 3) wrap, (-4, 2) sits on the unpaired mode)."""
    N = 8
    op = O.Operator(2, N, math.pi, S_TRUNC, 0, 1.0, wrap=1)
    G = np.zeros((N, N), dtype=np.complex128)
    k = np.array(k0)
    G[tuple(k + N // 2)] = 1.0
    fast = _appendix(op, G)
    n = _wrap(3 * k, N)
    a = _wrap(2 * k, N)
    expect = np.zeros_like(fast)
    expect[tuple(n + N // 2)] = op.beta_at(a, a)
    assert np.abs(fast - expect).max() <= 1e-13 * abs(op.beta_at(a, a))


def test_shift_identity_of_step_4():
    """g_{p,j}(x) = g_{p,0}(x - j): the inverse transform of alpha_p(k) e^{-2i pi k.j/N} is the
    node's transform shifted by j (the identity behind the "shifted" operation count)."""
    N = 6
    op = O.Operator(2, N, math.pi, S_TRUNC, 0, 1.0, wrap=1)
    al, _ = op.alpha_tables()
    a = np.fft.ifftshift(AP.alpha_on_IN(al, 2, N)[3])
    g0 = np.fft.ifftn(a) * N * N
    for j in [(1, 0), (2, 5), (4, 3)]:
        ph = np.exp(-2j * np.pi * (np.arange(N)[:, None] * j[0] + np.arange(N)[None, :] * j[1]) / N)
        gj = np.fft.ifftn(a * ph) * N * N
        assert np.allclose(gj, np.roll(g0, j, axis=(0, 1)), rtol=0, atol=1e-14 * np.abs(g0).max())


def test_operation_counts():
    """The direct counts against enumeration; the Appendix's transform count (4 per node and grid
    point as printed, 2 with the shift identity)."""
    c = AP.appendix_operation_counts(2, 4, 8)
    assert c["direct_circular_triples"] == 16 ** 3
    lin = sum(1 for k, l, m in itertools.product(range(-2, 2), repeat=3) if -2 <= k + l + m < 2) ** 2
    assert c["direct_linear_triples"] == lin
    assert c["appendix_transforms"] == 4 * 8 * 16
    assert c["appendix_butterflies"] == 4 * 8 * 16 * (8 * 4)
    assert c["shifted_transforms"] == 2 * 8 * 16 + 2 * 8
    assert AP.appendix_operation_counts(3, 6, 9)["appendix_butterflies"] is None
