"""FP64 oracle of the Appendix's evaluation of Q_{1,q} by discrete transforms (Mouton & Rey,
Appendix A, "Fast evaluation of the collision kernel").

TEST INFRASTRUCTURE ONLY: the test suite is the only caller.  The product library never imports
this module, and it imports nothing from the product library.

The Appendix rewrites the cubic sum Q^_{1,q}(G)_n = sum_{k+l+m=n} beta(k+m, l+m) G^_k G^_l G^_m of
the Lemma (Sec. 2.3) in four steps:

1. beta(a, b) = C sum_p alpha_p(a) alpha'_p(b) (Sec. 2.5, eq. betadD); the oracle's alpha tables
   carry C and the quadrature weights, so here beta(a, b) = sum_p alpha_p(a) alpha'_p(b);
2. with k + m = n - l and l + m = n - k, and the change of summation index k -> n - k, l -> n - l:
   Q^_n = sum_p sum_{k,l} alpha_p(l) alpha'_p(k) G^_{n-k} G^_{n-l} G^_{k+l-n};
3. G^_{k+l-n} is written through the grid values, G^_q = N^{-d} sum_j G_j e^{-2i pi q.j/N}, so that
   the sums over k and l separate for each grid point j;
4. for each node p and grid point j, g_{p,j} and g'_{p,j} are the inverse transforms of
   alpha_p(k) e^{-2i pi k.j/N} and alpha'_p(k) e^{-2i pi k.j/N}; the two bracketed sums are the modes
   n of the products g_{p,j} G_h and g'_{p,j} G_h, and
   Q^_n = N^{-d} sum_p sum_j G_j e^{2i pi n.j/N} (g_{p,j} G_h)^_n (g'_{p,j} G_h)^_n.

Every index is taken modulo N (the transforms are periodic), so the result is the cubic sum with
the CIRCULAR truncation: n, m = n - k - l and the kernel-mode arguments k + m, l + m reduced into
I_N.  The Appendix prints the exponent of step 3 as (k - l - n) and the normalisation as 1/N; the
steps after it need (k + l - n) and N^{-d}, which is what is used here.

The transforms are numpy's FFTs, a library primitive for step 4's "inverse Fourier transform" and
the modes of a grid function; nothing else is fused or reordered.  Arrays of modes and of grid
values are indexed as in the rest of the oracle: row-major over [-N/2, N/2)^d, offset N/2.
"""
from __future__ import annotations

import numpy as np


def _to_fft_order(a: np.ndarray) -> np.ndarray:
    """Row-major over I_N = [-N/2, N/2)^d (offset N/2) -> numpy's FFT order (index k mod N)."""
    return np.fft.ifftshift(a)


def _from_fft_order(a: np.ndarray) -> np.ndarray:
    return np.fft.fftshift(a)


def alpha_on_IN(alpha_ext: np.ndarray, d: int, N: int) -> np.ndarray:
    """Restrict alpha tables over the extended box [-N, N-1]^d (shape (P, (2N)^d), row-major, offset
    N) to I_N: shape (P,) + (N,)*d, row-major with offset N/2."""
    P = alpha_ext.shape[0]
    a = alpha_ext.reshape((P,) + (2 * N,) * d)
    sl = (slice(None),) + (slice(N // 2, N // 2 + N),) * d
    return np.ascontiguousarray(a[sl])


def q1q_appendix(Ghat: np.ndarray, alpha: np.ndarray, alphap: np.ndarray) -> np.ndarray:
    """Q^_{1,q}(G_h, G_h, G_h)_n for every n in I_N by the four steps of the Appendix.

    Ghat: complex modes, shape (N,)*d over I_N.  alpha, alphap: shape (P,) + (N,)*d, the factors
    of eq. betadD on I_N with C folded in.  Returns complex modes, shape (N,)*d.
    """
    Ghat = np.asarray(Ghat, dtype=np.complex128)
    d, N = Ghat.ndim, Ghat.shape[0]
    nm = N ** d
    axes = tuple(range(1, d + 1))
    # grid values G_j = sum_k G^_k e^{2i pi k.j/N} (the inverse of step 3's transform)
    Gj = np.fft.ifftn(_to_fft_order(Ghat)) * nm                      # FFT order over j
    # e^{-2i pi k.j/N} for every grid point j (rows, FFT order) and mode k (columns, FFT order)
    grids = np.meshgrid(*([np.arange(N)] * d), indexing="ij")
    pos = np.stack([g.reshape(-1) for g in grids], -1)               # (nm, d) index mod N
    phase_kj = np.exp(-2j * np.pi * (pos @ pos.T) / N)               # [j, k]
    Q = np.zeros((N,) * d, dtype=np.complex128)                      # FFT order over n
    for p in range(alpha.shape[0]):
        a = _to_fft_order(alpha[p]).reshape(-1)
        ap = _to_fft_order(alphap[p]).reshape(-1)
        # step 4: the modes of g_{p,j} and g'_{p,j}, one row per grid point j
        gh = (phase_kj * a[None, :]).reshape((nm,) + (N,) * d)
        ghp = (phase_kj * ap[None, :]).reshape((nm,) + (N,) * d)
        g = np.fft.ifftn(gh, axes=axes) * nm                         # g_{p,j}(x)
        gp = np.fft.ifftn(ghp, axes=axes) * nm
        # modes n of the products with G_h: (g_{p,j} G_h)^_n = N^{-d} sum_x g G e^{-2i pi n.x/N}
        A = np.fft.fftn(g * Gj[None], axes=axes) / nm
        Ap = np.fft.fftn(gp * Gj[None], axes=axes) / nm
        # N^{-d} sum_j G_j e^{2i pi n.j/N} A A'
        w = (Gj.reshape(-1)[:, None] * np.conj(phase_kj)).reshape((nm,) + (N,) * d)
        Q += (w * A * Ap).sum(axis=0) / nm
    return _from_fft_order(Q)


def appendix_operation_counts(d: int, N: int, P: int) -> dict:
    """Complex operations of one evaluation of Q^_{1,q}, for comparing the Appendix's route with
    the direct sums (Remark rem:computComplexity): the direct CIRCULAR sum has N^{2d} triples per
    output; the Appendix as printed needs, per node p and grid point j, two inverse and two forward
    transforms of N^d points (radix-2 cost (N^d / 2) log2(N^d) butterflies each) and 3 N^d
    products.  The inverse transforms are shifts, g_{p,j}(x) = g_{p,0}(x - j), so with g_{p,0} and
    g'_{p,0} formed once per node only the two forward transforms remain ("shifted")."""
    nm = N ** d
    butterflies = nm // 2 * int(round(np.log2(nm))) if (N & (N - 1)) == 0 else None
    return {
        "direct_circular_triples": nm ** 3,
        "direct_linear_triples": (2 * (N ** 3 - N) // 3) ** d,
        "appendix_transforms": 4 * P * nm,
        "appendix_butterflies": None if butterflies is None else 4 * P * nm * butterflies,
        "shifted_transforms": 2 * P * nm + 2 * P,
        "shifted_butterflies": None if butterflies is None else (2 * P * nm + 2 * P) * butterflies,
        "appendix_products": 3 * P * nm * nm,
    }
