"""FP64 CPU oracle for the Fourier-Galerkin Boltzmann-Nordheim collision operator.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library never
imports this package, and this package never imports the product library.

The arithmetic lives in ``bn_oracle.c`` (plain C, FP64, OpenMP over output
modes); this module only marshals numpy arrays through ctypes.  Every function
follows the paper (Mouton & Rey, arXiv:2110.13735) as cited in the C source:
the Lemma of Sec. 2.3 as a direct sum, the kernel modes of Sec. 2.5 (eq. betadD),
the discrete transform of Sec. 3.3 step 2(a) and the classical scaling of
Sec. 3.2.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bn_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libbn_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``bn_oracle.c`` into ``oracle/_build/libbn_oracle.so`` with gcc."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", _LIB_PATH, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int), ("N", ctypes.c_int), ("T", ctypes.c_double), ("R", ctypes.c_double),
        ("kernel", ctypes.c_int), ("eps", ctypes.c_double), ("M", ctypes.c_int),
        ("M1", ctypes.c_int), ("M2", ctypes.c_int), ("c_phi", ctypes.c_double), ("quad3d", ctypes.c_int),
        ("Q", ctypes.c_int), ("wrap", ctypes.c_int),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.ora_num_terms.argtypes = [P]
        _lib.ora_alpha_tables.argtypes = [P, dp, dp]
        _lib.ora_beta_table.argtypes = [P, dp]
        _lib.ora_dft_forward.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        _lib.ora_dft_inverse_real.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        _lib.ora_collision_modes.argtypes = [P, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        _lib.ora_collision_modes_onthefly.argtypes = [P, dp, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
        ip = ctypes.POINTER(ctypes.c_int)
        _lib.ora_collision_modes_at.argtypes = [P, dp, dp, dp, ip, ctypes.c_int, dp, dp, dp, dp]
        _lib.ora_conserve.argtypes = [P, dp]
        _lib.ora_eval_collision_onthefly.argtypes = [P, dp, dp, dp, dp, dp, dp, dp]
        _lib.ora_scale.argtypes = [P]
        _lib.ora_scale.restype = ctypes.c_double
        _lib.ora_eval_collision.argtypes = [P, dp, dp, dp, dp, dp, dp]
        _lib.ora_step.argtypes = [P, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        _lib.ora_moments.argtypes = [P, dp, dp]
        _lib.ora_num_threads.restype = ctypes.c_int
        _lib.ora_set_threads.argtypes = [ctypes.c_int]
    return _lib


def _ptr(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return _load().ora_num_threads()


def set_threads(n: int) -> None:
    _load().ora_set_threads(int(n))


@dataclass
class Operator:
    """One collision operator: dimension, modes, box, truncation, kernel, eps.

    ``T`` is the velocity box half-width (the paper's L), ``R`` the truncation
    radius in velocity units (the paper's S = R, Sec. 4.1), ``kernel`` 0 for
    Maxwell molecules (2-D) and 1 for hard spheres (3-D, and 2-D by reading r5 of
    the C source with ``Q`` Gauss-Legendre points per radius), ``eps`` = +1
    bosons, -1 fermions, 0 classical (alpha = -eps in the paper's notation),
    ``wrap`` 0 for the Lemma's LINEAR truncation, 1 for the CIRCULAR variant
    (reading r6 of the C source).  Angular points: M = 2N (2-D), M1 = M2 = N/2 (3-D)
    unless given.
    """
    d: int
    N: int
    T: float
    R: float
    kernel: int
    eps: float
    M: int = 0
    M1: int = 0
    M2: int = 0
    c_phi: float = 0.0
    quad3d: int = 0
    Q: int = 0
    wrap: int = 0

    def __post_init__(self):
        if self.Q == 0:
            self.Q = self.N + 8
        if self.M == 0:
            self.M = 2 * self.N
        if self.M1 == 0:
            self.M1 = self.N // 2
        if self.M2 == 0:
            self.M2 = self.N // 2
        if self.c_phi == 0.0:
            self.c_phi = 1.0 / (2 * math.pi) if self.d == 2 else 1.0 / (4 * math.pi)
        self._beta = None
        self._alpha = None

    # full kernel-mode tables above this many entries are not formed; beta is then
    # evaluated on demand from the alpha tables (the sum of eq. betadD); in 3-D the
    # on-demand sum is also the faster one beyond N = 8
    TABLE_LIMIT = {2: 1 << 29, 3: 1 << 25}

    @property
    def use_table(self) -> bool:
        return (2 * self.N) ** (2 * self.d) <= self.TABLE_LIMIT[self.d]

    def _alpha_cached(self):
        if self._alpha is None:
            al, ap = self.alpha_tables()
            self._alpha = (np.ascontiguousarray(al.reshape(-1)), np.ascontiguousarray(ap.reshape(-1)))
        return self._alpha

    def _p(self):
        return _Params(self.d, self.N, self.T, self.R, self.kernel, self.eps, self.M, self.M1,
                       self.M2, self.c_phi, self.quad3d, self.Q, self.wrap)

    @property
    def n_modes(self) -> int:
        return self.N ** self.d

    @property
    def gamma(self) -> int:
        return 1 if self.kernel == 1 else 0

    def scale(self) -> float:
        p = self._p()
        return _load().ora_scale(ctypes.byref(p))

    def alpha_tables(self):
        lib = _load()
        p = self._p()
        P = lib.ora_num_terms(ctypes.byref(p))
        nE = (2 * self.N) ** self.d
        al = np.zeros(P * nE)
        ap = np.zeros(P * nE)
        lib.ora_alpha_tables(ctypes.byref(p), _ptr(al), _ptr(ap))
        return al.reshape(P, nE), ap.reshape(P, nE)

    def beta(self) -> np.ndarray:
        """beta[ia, ib] over the extended box a, b in [-N, N-1]^d (row-major, a+N)."""
        if self._beta is None:
            nE = (2 * self.N) ** self.d
            b = np.zeros(nE * nE)
            p = self._p()
            if _load().ora_beta_table(ctypes.byref(p), _ptr(b)) != 0:
                raise MemoryError("oracle beta table allocation failed")
            self._beta = b.reshape(nE, nE)
        return self._beta

    def beta_at(self, a, b) -> float:
        """beta(a, b) for integer vectors a, b in [-N, N-1]^d."""
        E = 2 * self.N
        ia = 0
        ib = 0
        for x, y in zip(a, b):
            ia = ia * E + (int(x) + self.N)
            ib = ib * E + (int(y) + self.N)
        return float(self.beta()[ia, ib])

    def collision_modes(self, Ghat: np.ndarray, n_lo: int | None = None, n_cnt: int | None = None):
        """Lemma of Sec. 2.3 on the output box [n_lo, n_lo+n_cnt)^d.

        Returns (Qhat, gain, loss, cubic), each complex of shape (n_cnt,)*d.
        """
        if n_lo is None:
            n_lo = -self.N // 2
        if n_cnt is None:
            n_cnt = self.N
        G = np.ascontiguousarray(np.asarray(Ghat, dtype=np.complex128).reshape(-1))
        assert G.size == self.n_modes
        Gd = G.view(np.float64)
        nOut = n_cnt ** self.d
        outs = [np.zeros(2 * nOut) for _ in range(4)]
        p = self._p()
        if self.use_table:
            beta = self.beta()
            _load().ora_collision_modes(ctypes.byref(p), _ptr(beta.reshape(-1)), _ptr(Gd), int(n_lo), int(n_cnt),
                                        *[_ptr(o) for o in outs])
        else:
            al, ap = self._alpha_cached()
            _load().ora_collision_modes_onthefly(ctypes.byref(p), _ptr(al), _ptr(ap), _ptr(Gd), int(n_lo),
                                                 int(n_cnt), *[_ptr(o) for o in outs])
        shape = (n_cnt,) * self.d
        return tuple(o.view(np.complex128).reshape(shape) for o in outs)

    def collision_modes_at(self, Ghat: np.ndarray, nlist):
        """The Lemma's sums at the listed output modes (an (count, d) integer array of modes in
        I_N), beta on demand from the alpha tables.  Returns (Qhat, gain, loss, cubic), each a
        complex array of length count."""
        G = np.ascontiguousarray(np.asarray(Ghat, dtype=np.complex128).reshape(-1))
        assert G.size == self.n_modes
        nl = np.ascontiguousarray(np.asarray(nlist, dtype=np.int32).reshape(-1, self.d))
        assert np.all(nl >= -self.N // 2) and np.all(nl < self.N // 2)
        count = nl.shape[0]
        outs = [np.zeros(2 * count) for _ in range(4)]
        al, ap = self._alpha_cached()
        p = self._p()
        r = _load().ora_collision_modes_at(ctypes.byref(p), _ptr(al), _ptr(ap), _ptr(G.view(np.float64)),
                                           nl.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), int(count),
                                           *[_ptr(o) for o in outs])
        if r != 0:
            raise MemoryError("oracle alpha-table copy failed")
        return tuple(o.view(np.complex128) for o in outs)

    def conserve(self, Q: np.ndarray) -> np.ndarray:
        """The conservation projection Q - C^T (C C^T)^{-1} C Q onto zero mass, momentum and
        energy (C: the collision invariants 1, v, |v|^2 on the grid)."""
        out = np.ascontiguousarray(np.asarray(Q, dtype=np.float64).reshape(-1)).copy()
        assert out.size == self.n_modes
        p = self._p()
        _load().ora_conserve(ctypes.byref(p), _ptr(out))
        return out.reshape((self.N,) * self.d)

    def dft(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        out = np.zeros(2 * f.size)
        _load().ora_dft_forward(self.d, self.N, _ptr(f), _ptr(out))
        return out.view(np.complex128).reshape((self.N,) * self.d)

    def idft_real(self, Qhat: np.ndarray) -> np.ndarray:
        Q = np.ascontiguousarray(np.asarray(Qhat, dtype=np.complex128).reshape(-1)).view(np.float64)
        out = np.zeros(self.n_modes)
        _load().ora_dft_inverse_real(self.d, self.N, _ptr(np.ascontiguousarray(Q)), _ptr(out))
        return out.reshape((self.N,) * self.d)

    def eval_collision(self, f: np.ndarray, parts: bool = False):
        """Q_eps(f) at the grid velocities v_j = 2Tj/N (velocity units).

        With ``parts=True`` also returns (gain, loss, cubic_bracket) in velocity units.
        """
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        assert f.size == self.n_modes
        Q = np.zeros_like(f)
        p = self._p()
        g, l, c = (np.zeros_like(f), np.zeros_like(f), np.zeros_like(f)) if parts else (None, None, None)
        if self.use_table:
            beta = self.beta()
            _load().ora_eval_collision(ctypes.byref(p), _ptr(beta.reshape(-1)), _ptr(f), _ptr(Q), _ptr(g), _ptr(l),
                                       _ptr(c))
        else:
            al, ap = self._alpha_cached()
            _load().ora_eval_collision_onthefly(ctypes.byref(p), _ptr(al), _ptr(ap), _ptr(f), _ptr(Q), _ptr(g),
                                                _ptr(l), _ptr(c))
        shape = (self.N,) * self.d
        if parts:
            return Q.reshape(shape), g.reshape(shape), l.reshape(shape), c.reshape(shape)
        return Q.reshape(shape)

    def step(self, f: np.ndarray, dt: float, nsteps: int, integrator: int = 0) -> np.ndarray:
        """``nsteps`` steps of RK4 (integrator 0) or SSP-RK2 (1); returns the new state
        (needs the full kernel-mode table)."""
        y = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1)).copy()
        beta = self.beta()
        p = self._p()
        _load().ora_step(ctypes.byref(p), _ptr(beta.reshape(-1)), _ptr(y), float(dt), int(nsteps), int(integrator))
        return y.reshape((self.N,) * self.d)

    def moments(self, f: np.ndarray) -> np.ndarray:
        """[rho, rho*u (d), e, E_c, H, max f]."""
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        out = np.zeros(self.d + 5)
        p = self._p()
        _load().ora_moments(ctypes.byref(p), _ptr(f), _ptr(out))
        return out

    def velocities(self) -> np.ndarray:
        """Grid velocities v_j = 2Tj/N, j in I_N, shape (N,)*d + (d,)."""
        j = np.arange(-self.N // 2, self.N // 2)
        h = 2.0 * self.T / self.N
        grids = np.meshgrid(*([j * h] * self.d), indexing="ij")
        return np.stack(grids, axis=-1)
