"""Python binding of libbn (include/bn.h): argument marshalling only.

Every step of the collision operator and of the time stepping runs in the CUDA
library; this module converts numpy arrays / torch tensors to pointers and
statuses to exceptions.  Importing it does not need a GPU; creating a solver
does, and fails loudly when the library or the device is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbn.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "bn.h")

BN_OK = 0
STATUS = {0: "BN_OK", -1: "BN_ERR_ARG", -2: "BN_ERR_ALIAS", -3: "BN_ERR_NOMEM", -4: "BN_ERR_CUDA",
          -5: "BN_ERR_NONFINITE", -6: "BN_ERR_TIMEOUT", -7: "BN_ERR_STATE", -8: "BN_ERR_UNSUPPORTED"}
MAXWELL, HARD_SPHERE = 0, 1
FP64, MIXED = 0, 1


class BNError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("M1", ctypes.c_int), ("M2", ctypes.c_int), ("precision", ctypes.c_int),
                ("conserve", ctypes.c_int), ("c_phi", ctypes.c_double), ("integrator", ctypes.c_int),
                ("quad3d", ctypes.c_int), ("escalate_at", ctypes.c_double),
                ("mixed_rw", ctypes.c_int), ("mixed_variant", ctypes.c_int), ("wrap", ctypes.c_int),
                ("beta_resident", ctypes.c_int), ("beta_budget_mb", ctypes.c_longlong), ("pair_weights", ctypes.c_int),
                ("shard_index", ctypes.c_int), ("shard_count", ctypes.c_int), ("debug_wait_giveup", ctypes.c_int),
                ("beta_split", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("N", ctypes.c_int), ("T", ctypes.c_double), ("R", ctypes.c_double),
                ("kernel", ctypes.c_int), ("eps", ctypes.c_double), ("opt", Options), ("dt", ctypes.c_double),
                ("t_end", ctypes.c_double)]


_lib = None


def load(path: str | None = None):
    """Load libbn.so (built by ``paper_2110_13735_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libbn.so not found at {path}: run paper_2110_13735_gb300/build.py (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, dp, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t
    lib.bn_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.bn_options_bytes.restype = ctypes.c_size_t
    lib.bn_request_bytes.restype = ctypes.c_size_t
    lib.bn_create_solver.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_double, ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
    lib.bn_destroy_solver.argtypes = [vp]
    lib.bn_destroy_solver.restype = None
    lib.bn_set_state.argtypes = [vp, dp, sz]
    lib.bn_set_state_device.argtypes = [vp, vp, sz]
    lib.bn_get_state.argtypes = [vp, dp, sz]
    lib.bn_get_state_device.argtypes = [vp, vp, sz]
    lib.bn_eval_collision.argtypes = [vp, dp, sz]
    lib.bn_eval_collision_device.argtypes = [vp, vp, vp, sz]
    lib.bn_eval_collision_modes.argtypes = [vp, dp, sz]
    lib.bn_eval_collision_noalloc.argtypes = [vp, vp, vp, sz, vp]
    lib.bn_step_rk.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    lib.bn_moments.argtypes = [vp, dp, sz]
    lib.bn_work_counts.argtypes = [vp, dp, sz]
    lib.bn_precision_state.argtypes = [vp, ctypes.POINTER(ctypes.c_int), dp, dp]
    lib.bn_kernel_config.argtypes = [vp, dp, sz]
    lib.bn_rescale_set.argtypes = [vp, ctypes.c_double, ctypes.c_double, dp, sz, ctypes.c_double, ctypes.c_double]
    lib.bn_step_rescaled.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    lib.bn_step_rescaled_rk2.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    lib.bn_rescale_get.argtypes = [vp, dp, sz]
    lib.bn_equilibrium_temperature.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    ip = ctypes.POINTER(ctypes.c_int)
    lib.bn_plan_mixed2d.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, sz, ip]
    lib.bn_measure_fma_peak.argtypes = [ctypes.c_int, vp, dp, sz]
    lib.bn_plan_shards.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), sz]
    lib.bn_kernel_launches.argtypes = [vp]
    lib.bn_kernel_launches.restype = ctypes.c_longlong
    lib.bn_last_error.restype = ctypes.c_char_p
    lib.bn_profile_enable.argtypes = [vp, ctypes.c_int]
    lib.bn_profile_read.argtypes = [vp, dp, sz]
    lib.bn_profile_nd.argtypes = [vp, dp, sz]
    lib.bn_step_rk_batch.argtypes = [ctypes.POINTER(vp), ctypes.c_int, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.bn_server_create.argtypes = [sz, ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.bn_server_submit.argtypes = [vp, ctypes.POINTER(Request), dp, sz, ctypes.POINTER(ctypes.c_longlong)]
    lib.bn_server_poll.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int), dp, sz, dp, sz]
    lib.bn_server_wait_idle.argtypes = [vp, ctypes.c_double]
    lib.bn_server_stats.argtypes = [vp, dp, sz]
    lib.bn_server_last_error.restype = ctypes.c_char_p
    lib.bn_server_destroy.argtypes = [vp]
    lib.bn_server_destroy.restype = None
    _lib = lib
    return lib


def declared_symbols(header: str = HEADER):
    """Names of the functions declared in include/bn.h."""
    import re
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bn_[a-z_0-9]+)\s*\(", text)))


def _check(status: int):
    if status != BN_OK:
        msg = _lib.bn_last_error().decode() if _lib is not None else ""
        raise BNError(status, msg)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


PLAN_COLUMNS = ("ib", "orient", "J", "chunk", "units", "J2", "chunk2", "units2", "tail0", "base",
                "Lu", "Lw", "Su", "Sw")


def plan_mixed2d(N: int, rw: int = 8, oriented: bool = True, nblk: int = 456) -> np.ndarray:
    """The mixed 2-D kernel's host-side plan (include/bn.h: bn_plan_mixed2d): one row per work item
    in the order the CTAs take them, columns PLAN_COLUMNS.  Needs no GPU."""
    lib = load()
    n = ctypes.c_int()
    _check(lib.bn_plan_mixed2d(int(N), int(rw), int(bool(oriented)), int(nblk), None, 0, ctypes.byref(n)))
    out = np.zeros((n.value, len(PLAN_COLUMNS)), dtype=np.int32)
    _check(lib.bn_plan_mixed2d(int(N), int(rw), int(bool(oriented)), int(nblk),
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), out.size, ctypes.byref(n)))
    return out


def equilibrium_temperature(d: int, eps: float, rho: float, e: float):
    """(T, z) of the equilibrium with mass rho and internal energy e (include/bn.h:
    bn_equilibrium_temperature); host only."""
    lib = load()
    T, z = ctypes.c_double(), ctypes.c_double()
    _check(lib.bn_equilibrium_temperature(int(d), float(eps), float(rho), float(e), ctypes.byref(T), ctypes.byref(z)))
    return T.value, z.value


def options(M=0, M1=0, M2=0, precision=FP64, conserve=0, c_phi=0.0, integrator=0, quad3d=0,
            escalate_at=0.0, mixed_rw=0, mixed_variant=0, wrap=0, beta_resident=0, beta_budget_mb=0,
            pair_weights=0, shard_index=0, shard_count=0, debug_wait_giveup=0, beta_split=0) -> Options:
    o = Options()
    o.M, o.M1, o.M2, o.precision, o.conserve = M, M1, M2, precision, conserve
    o.c_phi, o.integrator, o.quad3d, o.escalate_at = c_phi, integrator, quad3d, escalate_at
    o.mixed_rw, o.mixed_variant = mixed_rw, mixed_variant
    o.wrap, o.beta_resident, o.beta_budget_mb, o.pair_weights = wrap, beta_resident, beta_budget_mb, pair_weights
    o.shard_index, o.shard_count, o.debug_wait_giveup = shard_index, shard_count, debug_wait_giveup
    o.beta_split = beta_split
    return o


class Solver:
    """One collision operator (d, N, T, R, kernel, eps) with its device state.

    ``stream`` may be a ``torch.cuda.Stream`` or a raw ``cudaStream_t`` integer.
    """

    def __init__(self, d, N, T, R, kernel=MAXWELL, eps=0.0, stream=None, **opts):
        lib = load()
        self.d, self.N, self.T, self.R, self.kernel, self.eps = int(d), int(N), float(T), float(R), int(kernel), float(eps)
        self.opts = options(**opts)
        raw = 0
        if stream is not None:
            raw = int(getattr(stream, "cuda_stream", stream))
        h = ctypes.c_void_p()
        _check(lib.bn_create_solver(self.d, self.N, self.T, self.R, self.kernel, self.eps, ctypes.byref(self.opts),
                                    ctypes.c_void_p(raw) if raw else None, ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def n_modes(self):
        return self.N ** self.d

    @property
    def shape(self):
        return (self.N,) * self.d

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.bn_destroy_solver(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, f):
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        _check(_lib.bn_set_state(self._h, _dptr(f), f.size))

    def set_state_device(self, f_dev):
        """f_dev: a contiguous float64 CUDA tensor with N^d entries."""
        _check(_lib.bn_set_state_device(self._h, ctypes.c_void_p(f_dev.data_ptr()), f_dev.numel()))

    def get_state(self, out: np.ndarray | None = None) -> np.ndarray:
        """The state on the host; into ``out`` (contiguous float64, N^d entries, e.g. pinned memory)
        when given, else into a new array."""
        if out is None:
            out = np.empty(self.n_modes)
        elif out.dtype != np.float64 or out.size != self.n_modes or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous float64 array of N^d entries")
        _check(_lib.bn_get_state(self._h, _dptr(out), out.size))
        return out.reshape(self.shape)

    def get_state_device(self, out_dev):
        _check(_lib.bn_get_state_device(self._h, ctypes.c_void_p(out_dev.data_ptr()), out_dev.numel()))

    def eval_collision(self) -> np.ndarray:
        out = np.empty(self.n_modes)
        _check(_lib.bn_eval_collision(self._h, _dptr(out), out.size))
        return out.reshape(self.shape)

    def eval_collision_modes(self) -> np.ndarray:
        """Q^_n, n in I_N^d (complex, shape (N,)*d), before the inverse transform and prefactor."""
        out = np.empty(2 * self.n_modes)
        _check(_lib.bn_eval_collision_modes(self._h, _dptr(out), out.size))
        return out.view(np.complex128).reshape(self.shape)

    def eval_collision_noalloc(self, f_dev, Q_dev, stream=None):
        """Q_eps(f_dev) into Q_dev without device allocation (include/bn.h: bn_eval_collision_noalloc)."""
        raw = int(getattr(stream, "cuda_stream", stream)) if stream is not None else 0
        _check(_lib.bn_eval_collision_noalloc(self._h, ctypes.c_void_p(f_dev.data_ptr()),
                                              ctypes.c_void_p(Q_dev.data_ptr()), f_dev.numel(),
                                              ctypes.c_void_p(raw) if raw else None))

    def eval_collision_device(self, f_dev, Q_dev):
        _check(_lib.bn_eval_collision_device(self._h, ctypes.c_void_p(f_dev.data_ptr()),
                                             ctypes.c_void_p(Q_dev.data_ptr()), f_dev.numel()))

    def step_rk(self, dt: float, nsteps: int):
        _check(_lib.bn_step_rk(self._h, float(dt), int(nsteps)))

    def moments(self) -> np.ndarray:
        out = np.empty(self.d + 6)
        _check(_lib.bn_moments(self._h, _dptr(out), out.size))
        return out

    def work_counts(self) -> np.ndarray:
        out = np.empty(4)
        _check(_lib.bn_work_counts(self._h, _dptr(out), out.size))
        return out

    def kernel_config(self):
        """(outputs per thread, CTAs per launch, oriented (0/1), tuner ms of the variants
        (8, 8 oriented, 16, 16 oriented))."""
        out = np.zeros(7)
        _check(_lib.bn_kernel_config(self._h, _dptr(out), 7))
        return int(out[0]), int(out[1]), int(out[2]), tuple(float(x) for x in out[3:])

    def rescale_set(self, L: float, omega: float, u, rho: float, e: float):
        """Velocity rescaling (include/bn.h: bn_rescale_set): the state is G on the xi grid of a T = pi solver."""
        uu = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(-1))
        _check(_lib.bn_rescale_set(self._h, float(L), float(omega), _dptr(uu), uu.size, float(rho), float(e)))

    def step_rescaled(self, dt: float, nsteps: int, rk2: bool = False):
        """nsteps forward Euler (bn_step_rescaled) or SSP-RK2 (bn_step_rescaled_rk2) rescaled steps."""
        fn = _lib.bn_step_rescaled_rk2 if rk2 else _lib.bn_step_rescaled
        _check(fn(self._h, float(dt), int(nsteps)))

    def rescale_state(self) -> dict:
        """{w, u, rho, e, T, z, t} of the rescaled solve (include/bn.h: bn_rescale_get)."""
        out = np.zeros(9)
        _check(_lib.bn_rescale_get(self._h, _dptr(out), 9))
        return {"w": out[0], "u": out[1:1 + self.d].copy(), "rho": out[4], "e": out[5], "T": out[6], "z": out[7],
                "t": out[8]}

    def precision_state(self):
        """(precision in use, time of the switch to FP64 or -1, max f after the last step)."""
        p, t, m = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        _check(_lib.bn_precision_state(self._h, ctypes.byref(p), ctypes.byref(t), ctypes.byref(m)))
        return p.value, t.value, m.value

    def kernel_launches(self) -> int:
        return int(_lib.bn_kernel_launches(self._h))

    def profile_enable(self, on: bool = True):
        _check(_lib.bn_profile_enable(self._h, int(bool(on))))

    def profile_nd(self):
        """Phase timing of the 3-D / CIRCULAR operator since the last read (include/bn.h:
        bn_profile_nd): dict of ms per phase, evaluations, rounds, Q_{1,q} terms, CTAs."""
        out = np.zeros(8)
        _check(_lib.bn_profile_nd(self._h, _dptr(out), 8))
        keys = ["pair_ms", "beta_ms", "sweep_ms", "tail_ms", "evals", "rounds", "terms", "ctas"]
        return dict(zip(keys, out.tolist()))

    def profile_read(self):
        """Dominant-kernel timing since the last read:
        (event ms total, event launches, device-stamp ms total, stamped launches)."""
        out = np.zeros(4)
        _check(_lib.bn_profile_read(self._h, _dptr(out), 4))
        return float(out[0]), int(out[1]), float(out[2]), int(out[3])


def plan_shards(d: int, N: int, count: int, wrap: int = 0) -> np.ndarray:
    """Output-plane ranges of `count` shards of one evaluation (include/bn.h: bn_plan_shards); no GPU."""
    lib = load()
    out = np.zeros(count + 1, dtype=np.int32)
    _check(lib.bn_plan_shards(int(d), int(N), int(wrap), int(count), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              out.size))
    return out


def measure_fma_peak(kind: int, stream=None):
    """Measured FMA rate of the current device (include/bn.h: bn_measure_fma_peak): kind 0 FP32,
    1 paired FP32, 2 FP64.  Returns (TFLOP/s, ms of the timed launch)."""
    lib = load()
    raw = int(getattr(stream, "cuda_stream", stream)) if stream is not None else 0
    out = np.zeros(3)
    _check(lib.bn_measure_fma_peak(int(kind), ctypes.c_void_p(raw) if raw else None, _dptr(out), 3))
    return float(out[0]), float(out[1])


def step_rk_batch(solvers, dts, nsteps: int):
    """Advance several solvers together (include/bn.h: bn_step_rk_batch); returns the failed index or -1."""
    lib = load()
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s.handle.value for s in solvers])
    d = np.ascontiguousarray(np.asarray(dts, dtype=np.float64))
    failed = ctypes.c_int(-1)
    st = lib.bn_step_rk_batch(hs, n, _dptr(d), int(nsteps), ctypes.byref(failed))
    _check(st)
    return failed.value


class Server:
    """Continuous-batching solve server (include/bn.h: bn_server_*)."""

    def __init__(self, device_bytes: int = 0, max_active: int = 64, stream=None):
        lib = load()
        raw = int(getattr(stream, "cuda_stream", stream)) if stream is not None else 0
        h = ctypes.c_void_p()
        st = lib.bn_server_create(int(device_bytes), int(max_active), ctypes.c_void_p(raw) if raw else None,
                                  ctypes.byref(h))
        if st != BN_OK:
            raise BNError(st, lib.bn_server_last_error().decode())
        self._h = h

    def _chk(self, st):
        if st != BN_OK:
            raise BNError(st, _lib.bn_server_last_error().decode())

    def submit(self, d, N, T, R, kernel, eps, f0, dt, t_end, **opts) -> int:
        r = Request()
        r.d, r.N, r.T, r.R, r.kernel, r.eps = int(d), int(N), float(T), float(R), int(kernel), float(eps)
        r.opt = options(**opts)
        r.dt, r.t_end = float(dt), float(t_end)
        f = np.ascontiguousarray(np.asarray(f0, dtype=np.float64).reshape(-1))
        rid = ctypes.c_longlong()
        self._chk(_lib.bn_server_submit(self._h, ctypes.byref(r), _dptr(f), f.size, ctypes.byref(rid)))
        return int(rid.value)

    def poll(self, rid: int, n_modes: int | None = None):
        """(state, result or None, (t_submit, t_admit, t_done, t_escalated)); state 0 queued, 1 running,
        2 done, 3 failed; t_escalated is the solve time of the switch to FP64, -1 if none."""
        state = ctypes.c_int()
        times = np.full(4, -1.0)
        out = np.empty(n_modes) if n_modes else None
        st = _lib.bn_server_poll(self._h, int(rid), ctypes.byref(state), _dptr(out) if out is not None else None,
                                 out.size if out is not None else 0, _dptr(times), 4)
        if st != BN_OK and state.value != 3:
            self._chk(st)
        return state.value, (out if state.value == 2 else None), tuple(times)

    def wait_idle(self, timeout: float = 600.0):
        self._chk(_lib.bn_server_wait_idle(self._h, float(timeout)))

    def stats(self):
        out = np.zeros(8)
        self._chk(_lib.bn_server_stats(self._h, _dptr(out), 8))
        keys = ["submitted", "admitted", "done", "failed", "ticks", "max_active", "bytes_in_use", "budget"]
        return dict(zip(keys, out.tolist()))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.bn_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
