"""Pins of the oracle's Lemma sums (LINEAR and CIRCULAR truncation) against discrete
convolutions computed with numpy's FFT, and of its on-demand kernel modes against its table.

With beta(a,b) = sum_p alpha_p(a) alpha'_p(b) (Sec. 2.5, eq. betadD), every sum of the Lemma
of Sec. 2.3 is a sum over the quadrature nodes of convolutions of pointwise products of the
modes G^ with the node functions alpha_p, alpha'_p (the route the Appendix takes for Q_{1,q}):

  gain(n)  = sum_p [(alpha_p G^) * (alpha'_p G^)](n)
  loss(n)  = [G^ * (beta(l,l) G^_l)](n)
  Q1q(n)   = sum_p sum_m G^_m [u_{p,m} * v_{p,m}](n - m),
             u_{p,m}(k) = alpha_p(k+m) G^_k,  v_{p,m}(l) = alpha'_p(l+m) G^_l
  Q2q(n)   = [G^ * S2](n),  S2(t) = sum_p [(alpha_p G^) * (alpha'_p G^)](t)
  Q3q(n)   = [G^ * S3](n),  S3(t) = sum_p alpha_p(t) [(alpha'_p G^) * G^](t)
  Q4q(n)   = [G^ * S4](n),  S4(t) = sum_p alpha'_p(t) [(alpha_p G^) * G^](t)

with * the linear convolution (zero-padded FFT) for the Lemma's LINEAR truncation, and the
cyclic convolution on I_N with every index sum reduced modulo N for the CIRCULAR variant.  The
oracle instead loops over the index pairs and triples with the four kernel-mode lookups per
term; the two share nothing but the alpha tables (pinned by the closed forms in
test_oracle_pins.py).  A wrong label, sign, index reduction or a dropped term changes these
sums far beyond the 1e-12 tolerance.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
from paper_2110_13735_gb300 import inputs as I

R6 = 6.0
T6 = I.box_half_width(R6)


def _random_modes(d, N, seed, support=None):
    """Hermitian-ish random G^ on I_N^d (complex; the sums do not need Hermitian symmetry)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((N,) * d) + 1j * rng.standard_normal((N,) * d)
    if support is not None:
        k = np.arange(-N // 2, N // 2)
        mask = np.ones((N,) * d, bool)
        for ax in range(d):
            sh = [1] * d
            sh[ax] = N
            mask &= (np.abs(k) <= support).reshape(sh)
        G = np.where(mask, G, 0.0)
    return G


def _ext_slice(tab, d, N, lo, cnt):
    """Rows of an alpha table ([P][(2N)^d], a + N row-major) restricted to the box [lo, lo+cnt)^d."""
    P = tab.shape[0]
    t = tab.reshape((P,) + (2 * N,) * d)
    idx = tuple([slice(None)] + [slice(lo + N, lo + N + cnt)] * d)
    return t[idx]


def _lin_conv(a, b, full=False):
    """Linear convolution of two arrays on I_N^d (offset -N/2): result on [-N, N-2]^d, shape
    (2N-1)^d (full: shape (2N)^d, the last position of each axis zero)."""
    d = a.ndim
    N = a.shape[0]
    s, ax = (2 * N,) * d, tuple(range(d))
    c = np.fft.ifftn(np.fft.fftn(a, s, ax) * np.fft.fftn(b, s, ax), axes=ax)
    return c if full else c[tuple([slice(0, 2 * N - 1)] * d)]   # position q <-> index q - N


def _cyc_conv(a, b):
    """Cyclic convolution on I_N^d (index k stored at k + N/2): same layout in and out."""
    fa = np.fft.fftn(np.fft.ifftshift(a))
    fb = np.fft.fftn(np.fft.ifftshift(b))
    return np.fft.fftshift(np.fft.ifftn(fa * fb))


def _fft_sums(op, G, wrap):
    d, N = op.d, op.N
    al, ap = op.alpha_tables()
    P = al.shape[0]
    h = N // 2
    AI = _ext_slice(al, d, N, -h, N)      # alpha_p on I_N
    BI = _ext_slice(ap, d, N, -h, N)      # alpha'_p on I_N
    conv = _cyc_conv if wrap else _lin_conv
    # gain and S2 share the same pair sum
    pair = sum(conv(AI[p] * G, BI[p] * G) for p in range(P))
    betadiag = np.einsum("p...,p...->...", AI, BI)          # beta(l, l), l in I_N
    loss_full = conv(G, betadiag * G)
    if wrap:
        A_t, B_t = AI, BI                                    # alpha at t in I_N (reduced sums)
    else:
        A_t = _ext_slice(al, d, N, -N, 2 * N - 1)            # alpha_p(t), t in [-N, N-2]^d
        B_t = _ext_slice(ap, d, N, -N, 2 * N - 1)
    S3 = sum(A_t[p] * conv(BI[p] * G, G) for p in range(P))
    S4 = sum(B_t[p] * conv(AI[p] * G, G) for p in range(P))
    S2 = pair

    def outer(S):
        """[G^ * S](n), n in I_N: linear (S on [-N, N-2]^d) or cyclic (S on I_N)."""
        if wrap:
            return _cyc_conv(G, S)
        s, ax = (3 * N,) * d, tuple(range(d))
        c = np.fft.ifftn(np.fft.fftn(G, s, ax) * np.fft.fftn(S, s, ax), axes=ax)   # q <-> index q - 3N/2
        return c[tuple([slice(N, 2 * N)] * d)]

    # Q1q: for each node p and each m, a convolution of the shifted node functions
    Q1q = np.zeros((N,) * d, complex)
    ms = np.stack(np.meshgrid(*([np.arange(-h, h)] * d), indexing="ij"), -1).reshape(-1, d)
    for m in ms:
        if G[tuple(m + h)] == 0:
            continue
        if wrap:
            sh = tuple(int(x) for x in m)
            for p in range(P):
                # alpha_p(<k + m>) for k in I_N: roll the I_N table by -m (cyclic)
                u = np.roll(AI[p], tuple(-x for x in sh), axis=tuple(range(d))) * G
                v = np.roll(BI[p], tuple(-x for x in sh), axis=tuple(range(d))) * G
                c = _cyc_conv(u, v)                              # index t = k + l (mod N)
                # Q1q(n) += G_m c(n - m): shift c by +m cyclically
                Q1q += G[tuple(m + h)] * np.roll(c, sh, axis=tuple(range(d)))
        else:
            lo = [int(x) - h for x in m]
            for p in range(P):
                t = al[p].reshape((2 * N,) * d)
                tp = ap[p].reshape((2 * N,) * d)
                idx = tuple(slice(l + N, l + N + N) for l in lo)   # k + m for k in I_N
                u = t[idx] * G
                v = tp[idx] * G
                c = _lin_conv(u, v, full=True)                   # position q <-> k + l = q - N
                # n - m = k + l  ->  n in I_N needs q = n - m + N
                sel = tuple(slice(-h - int(x) + N, h - int(x) + N) for x in m)
                Q1q += G[tuple(m + h)] * c[sel]
    if wrap:
        gain, loss = pair, loss_full
    else:
        sel = tuple([slice(N - h, N + h)] * d)                 # n in I_N
        gain, loss = pair[sel], loss_full[sel]
    cubic = Q1q + outer(S2) - outer(S3) - outer(S4)
    return gain, loss, cubic


CASES = [
    (2, 8, dict(M=16, kernel=0), 1.0),
    (2, 6, dict(M=12, kernel=1, Q=10), -1.0),
    (3, 4, dict(M1=3, M2=4, kernel=1), 1.0),
]


@pytest.mark.parametrize("wrap", [0, 1])
@pytest.mark.parametrize("d,N,kw,eps", CASES)
def test_lemma_sums_equal_fft_convolutions(d, N, kw, eps, wrap):
    kw = dict(kw)
    kernel = kw.pop("kernel")
    op = O.Operator(d, N, T6, R6, kernel, eps, wrap=wrap, **kw)
    G = _random_modes(d, N, 11 + d + N + wrap)
    Qh, gain, loss, cubic = op.collision_modes(G)
    g_f, l_f, c_f = _fft_sums(op, G, wrap)
    scale = np.abs(gain).max()
    assert np.abs(gain - g_f).max() <= 1e-12 * scale
    assert np.abs(loss - l_f).max() <= 1e-12 * scale
    assert np.abs(cubic - c_f).max() <= 1e-12 * np.abs(c_f).max()
    assert np.abs(Qh - (gain - loss + eps * cubic)).max() <= 1e-13 * scale


def test_circular_equals_linear_when_nothing_wraps():
    """With G^ supported in |k_i| <= 2 at N = 16 every sum k+l+m and every kernel-mode argument
    stays inside I_N: the CIRCULAR variant then has exactly the LINEAR terms."""
    G = _random_modes(2, 16, 5, support=2)
    ops = [O.Operator(2, 16, T6, R6, 0, 1.0, M=16, wrap=w) for w in (0, 1)]
    lin = ops[0].collision_modes(G)
    cir = ops[1].collision_modes(G)
    for a, b in zip(lin, cir):
        assert np.abs(a - b).max() <= 1e-14 * np.abs(lin[1]).max()


def test_circular_differs_when_sums_wrap():
    G = _random_modes(2, 8, 6)
    lin = O.Operator(2, 8, T6, R6, 0, 1.0, M=16).collision_modes(G)[3]
    cir = O.Operator(2, 8, T6, R6, 0, 1.0, M=16, wrap=1).collision_modes(G)[3]
    assert np.abs(lin - cir).max() > 1e-3 * np.abs(lin).max()


@pytest.mark.parametrize("d,N,kw", [(2, 8, dict(M=16)), (3, 4, dict(M1=3, M2=4))])
@pytest.mark.parametrize("wrap", [0, 1])
def test_on_demand_kernel_modes_equal_table(d, N, kw, wrap):
    """The on-demand sum over the nodes (used for sizes whose table does not fit) gives the
    table's kernel modes up to the rounding order of that sum, at every output and at a list."""
    op = O.Operator(d, N, T6, R6, 0 if d == 2 else 1, 1.0, wrap=wrap, **kw)
    assert op.use_table
    G = _random_modes(d, N, 21 + d)
    Gf = np.ascontiguousarray(G.reshape(-1))
    outs_t = [np.zeros(2 * N ** d) for _ in range(4)]
    outs_f = [np.zeros(2 * N ** d) for _ in range(4)]
    lib = O._load()
    p = op._p()
    import ctypes
    lib.ora_collision_modes(ctypes.byref(p), O._ptr(op.beta().reshape(-1)), O._ptr(Gf.view(np.float64)), -N // 2, N,
                            *[O._ptr(o) for o in outs_t])
    al, ap = op._alpha_cached()
    lib.ora_collision_modes_onthefly(ctypes.byref(p), O._ptr(al), O._ptr(ap), O._ptr(Gf.view(np.float64)), -N // 2,
                                     N, *[O._ptr(o) for o in outs_f])
    scale = np.abs(outs_t[1]).max()
    for a, b in zip(outs_t, outs_f):
        assert np.abs(a - b).max() <= 1e-13 * scale
    # the list form at a few modes, including the corners of I_N
    h = N // 2
    nl = np.array([[-h] * d, [h - 1] * d, [0] * d, [-h] + [h - 1] * (d - 1)], dtype=np.int32)
    at = op.collision_modes_at(G, nl)
    flat = [int(np.ravel_multi_index(tuple(n + h), (N,) * d)) for n in nl]
    for a, b in zip(at, outs_t):
        bc = b.view(np.complex128)[flat]
        assert np.abs(a - bc).max() <= 1e-13 * scale
