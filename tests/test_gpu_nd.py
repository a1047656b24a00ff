"""GPU parity of the 3-D operator and of the CIRCULAR truncation (kernel-mode slices recomputed from
the quadrature factors at every evaluation) against the FP64 oracle, through the C ABI.

Error measure: e_Q = ||Q^_gpu - Q^_oracle||_2 / ||Q^{1c}_oracle||_2 over the compared modes (the
classical gain term does not vanish near equilibrium).  Bars: FP64 1e-12; mixed precision (FP32
kernel-mode slices and sums with compensated accumulation, FP64 elsewhere) 2e-6, the measured value
printed per case.

Sizes: every output at 3-D N <= 16; at N = 32 the oracle evaluates sampled modes (the corners of
I_N, edges and the centre) one by one; at N = 32 and 48 with the default quadrature a state whose
modes are a few random trigonometric modes (the GPU still evaluates every term; the oracle skips
exact zeros) is compared on several hundred sampled modes.  FP64 at N = 48 is not run here: one
evaluation takes about 26 minutes on a GB300 (4e14 terms at the FP64 rate).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2110_13735_gb300 import inputs as I

pytestmark = pytest.mark.gpu

R6 = 6.0
T6 = I.box_half_width(R6)


@pytest.fixture(scope="module")
def B():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_13735_gb300 import build as BUILD
    BUILD.build()
    from paper_2110_13735_gb300 import bn
    bn.load()
    return bn


def _f(d, N, seed):
    rng = np.random.Generator(np.random.PCG64(I.SEED + 100 + seed))
    base = I.two_gaussians(d, N, T6, 0.9, (1.5, 0.0, 0.0)[:d] if d == 3 else (2.0, 1.0), 0.8)
    return base * (1.0 + 0.2 * rng.uniform(size=(N,) * d))


def _kernel(B, d):
    return B.HARD_SPHERE if d == 3 else B.MAXWELL


def _gpu_modes(B, d, N, eps, f, precision, **kw):
    prec = B.MIXED if precision == "mixed" else B.FP64
    with B.Solver(d, N, T6, R6, _kernel(B, d), eps, precision=prec, **kw) as s:
        s.set_state(f)
        return s.eval_collision_modes()


def _e(a, b, gain):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(gain.ravel()))


def _bar(precision):
    return 1e-12 if precision == "fp64" else 2e-6


# ------------------------------------------------------------------ 3-D LINEAR, every output
@pytest.mark.parametrize("N,eps,precision,M", [(4, 1.0, "fp64", 4), (6, -1.0, "fp64", 4), (8, 1.0, "fp64", 4),
                                               (8, -1.0, "mixed", 4), (12, 1.0, "fp64", 4), (12, -1.0, "mixed", 4),
                                               (16, 1.0, "mixed", 2), (16, -1.0, "fp64", 2)])
def test_3d_every_output(B, N, eps, precision, M):
    f = _f(3, N, N)
    ora = O.Operator(3, N, T6, R6, 1, eps, M1=M, M2=M)
    G = ora.dft(f)
    Qo, gain, _, _ = ora.collision_modes(G)
    Qg = _gpu_modes(B, 3, N, eps, f, precision, M1=M, M2=M)
    err = _e(Qg, Qo, gain)
    print(f"3-D N={N} eps={eps} {precision}: e_Q = {err:.3e}")
    assert err <= _bar(precision)


def _corner_and_sample_modes(d, N, count, seed):
    h = N // 2
    corners = np.array(np.meshgrid(*([[-h, h - 1]] * d), indexing="ij")).reshape(d, -1).T
    rng = np.random.Generator(np.random.PCG64(I.SEED + seed))
    edges = np.array([[-h, 0, h - 1][:d], [h - 1, -h, 0][:d], [0] * d, [-1] * d, [1 - h] + [h - 2] * (d - 1)])
    rnd = rng.integers(-h, h, size=(count, d))
    return np.unique(np.concatenate([corners, edges, rnd]), axis=0).astype(np.int32)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_3d_n32_sampled_modes(B, precision):
    """3-D N = 32 (dense state): the corners of I_N, edges, the centre and random modes."""
    N, eps, M = 32, -1.0, 2
    f = _f(3, N, 32)
    ora = O.Operator(3, N, T6, R6, 1, eps, M1=M, M2=M)
    G = ora.dft(f)
    nl = _corner_and_sample_modes(3, N, 6, 1)
    Qo, gain, _, _ = ora.collision_modes_at(G, nl)
    Qg = _gpu_modes(B, 3, N, eps, f, precision, M1=M, M2=M)
    h = N // 2
    Qg_s = np.array([Qg[tuple(n + h)] for n in nl])
    err = _e(Qg_s, Qo, gain)
    print(f"3-D N=32 sampled ({len(nl)} modes) {precision}: e_Q = {err:.3e}")
    assert err <= _bar(precision)


def _sparse_state(d, N, K, seed):
    """A real state whose modes are K random modes (and their conjugates) away from -N/2."""
    rng = np.random.Generator(np.random.PCG64(I.SEED + seed))
    h = N // 2
    G = np.zeros((N,) * d, complex)
    for _ in range(K):
        k = rng.integers(-h + 1, h, size=d)
        c = (rng.standard_normal() + 1j * rng.standard_normal()) * np.exp(-0.02 * float(k @ k))
        G[tuple(k + h)] += c
        G[tuple(-k + h)] += np.conj(c)
    # f_j = sum_k G_k e^{2 i pi k.j / N}, real by the conjugate pairs
    Gs = np.fft.ifftshift(G)
    f = np.fft.fftshift(np.fft.ifftn(Gs)).real * N ** d
    return f, G


@pytest.mark.parametrize("N", [32, 48])
def test_3d_sparse_modes_default_quadrature(B, N):
    """3-D N = 32 and 48, default quadrature (M1 = M2 = N/2), mixed precision: a state made of a
    few modes; every GPU term is still evaluated.  Compared on the corners and 400 sampled modes.
    The gain term of such a state vanishes at most sampled modes, so the error is normalised by
    ||Q^_oracle|| over the compared modes instead."""
    eps = 1.0
    f, G = _sparse_state(3, N, 12, N)
    ora = O.Operator(3, N, T6, R6, 1, eps)
    nl = _corner_and_sample_modes(3, N, 400, N)
    Qo, gain, _, _ = ora.collision_modes_at(G, nl)
    Qg = _gpu_modes(B, 3, N, eps, f, "mixed")
    h = N // 2
    Qg_s = np.array([Qg[tuple(n + h)] for n in nl])
    err = _e(Qg_s, Qo, Qo)
    print(f"3-D N={N} sparse state, {len(nl)} modes, mixed: ||dQ^|| / ||Q^|| = {err:.3e}")
    assert err <= 2e-6


# ------------------------------------------------------------------ CIRCULAR truncation
@pytest.mark.parametrize("d,N,eps,precision", [(2, 8, 1.0, "fp64"), (2, 16, -1.0, "fp64"), (2, 16, 1.0, "mixed"),
                                               (2, 32, 1.0, "mixed"), (2, 24, 0.0, "fp64"), (3, 4, 1.0, "fp64"),
                                               (3, 6, -1.0, "mixed"), (3, 8, 1.0, "fp64")])
def test_circular_every_output(B, d, N, eps, precision):
    f = _f(d, N, 7 + N)
    kw = dict(M=2 * N) if d == 2 else dict(M1=4, M2=4)
    ora = O.Operator(d, N, T6, R6, 0 if d == 2 else 1, eps, wrap=1, **kw)
    G = ora.dft(f)
    Qo, gain, _, _ = ora.collision_modes(G)
    Qg = _gpu_modes(B, d, N, eps, f, precision, wrap=1, **kw)
    err = _e(Qg, Qo, gain)
    print(f"CIRCULAR d={d} N={N} eps={eps} {precision}: e_Q = {err:.3e}")
    assert err <= _bar(precision)


def test_circular_differs_from_linear_on_the_gpu(B):
    f = _f(2, 16, 3)
    a = _gpu_modes(B, 2, 16, 1.0, f, "fp64")
    b = _gpu_modes(B, 2, 16, 1.0, f, "fp64", wrap=1)
    assert np.abs(a - b).max() > 1e-6 * np.abs(a).max()


# ------------------------------------------------------------------ 3-D: eps = 0, projection, time steps
def test_3d_classical_and_conservation_projection(B):
    """eps = 0 (quadratic part only) and the conservation projection against the oracle's
    projection of its own operator."""
    N = 8
    f = _f(3, N, 5)
    for eps in (0.0, 1.0):
        ora = O.Operator(3, N, T6, R6, 1, eps, M1=4, M2=4)
        Qo, gain, _, _ = ora.eval_collision(f, parts=True)
        Qp = ora.conserve(Qo)
        with B.Solver(3, N, T6, R6, B.HARD_SPHERE, eps, M1=4, M2=4, conserve=1) as s:
            s.set_state(f)
            Qg = s.eval_collision()
        err = _e(Qg, Qp, gain)
        print(f"3-D N=8 eps={eps} projected: e_Q = {err:.3e}")
        assert err <= 1e-12


def test_2d_conservation_projection_parity(B):
    N, eps = 16, -1.0
    f = _f(2, N, 9)
    for precision, bar in (("fp64", 1e-12), ("mixed", 2e-6)):
        ora = O.Operator(2, N, T6, R6, 0, eps, M=2 * N)
        Qo, gain, _, _ = ora.eval_collision(f, parts=True)
        Qp = ora.conserve(Qo)
        prec = B.MIXED if precision == "mixed" else B.FP64
        with B.Solver(2, N, T6, R6, B.MAXWELL, eps, precision=prec, conserve=1) as s:
            s.set_state(f)
            Qg = s.eval_collision()
        assert _e(Qg, Qp, gain) <= bar


@pytest.mark.parametrize("precision,integrator", [("fp64", 0), ("mixed", 0), ("fp64", 1)])
def test_3d_steps(B, precision, integrator):
    N, eps, dt = 8, 1.0, 0.01
    f = _f(3, N, 11)
    ora = O.Operator(3, N, T6, R6, 1, eps, M1=4, M2=4)
    f_o = ora.step(f, dt, 2, integrator)
    prec = B.MIXED if precision == "mixed" else B.FP64
    with B.Solver(3, N, T6, R6, B.HARD_SPHERE, eps, precision=prec, M1=4, M2=4, integrator=integrator) as s:
        s.set_state(f)
        s.step_rk(dt, 2)
        f_g = s.get_state()
    err = float(np.linalg.norm(f_g - f_o) / np.linalg.norm(f_o))
    print(f"3-D N=8 two steps ({precision}, integrator {integrator}): e_f = {err:.3e}")
    assert err <= (1e-12 if precision == "fp64" else 1e-7)


# ------------------------------------------------------------------ plan variants: rounds, resident, determinism
def test_3d_rounds_resident_and_determinism(B):
    """The same operator with the slices produced once and kept, recomputed per evaluation in
    one round, and recomputed in many small rounds (a 1 MiB slice budget): the first two are
    bitwise equal (same slices, same item order), the third within rounding; repeated
    evaluations are bitwise equal."""
    N, eps = 12, -1.0
    f = _f(3, N, 13)
    for precision, tol in (("mixed", 1e-6), ("fp64", 1e-13)):
        a = _gpu_modes(B, 3, N, eps, f, precision, M1=4, M2=4)
        b = _gpu_modes(B, 3, N, eps, f, precision, M1=4, M2=4, beta_resident=1)
        assert np.array_equal(a, b)
        prec = B.MIXED if precision == "mixed" else B.FP64
        with B.Solver(3, N, T6, R6, B.HARD_SPHERE, eps, precision=prec, M1=4, M2=4, beta_budget_mb=1) as s:
            s.set_state(f)
            c1 = s.eval_collision_modes()
            c2 = s.eval_collision_modes()
        assert np.array_equal(c1, c2)
        assert np.abs(c1 - a).max() <= tol * np.abs(a).max()


@pytest.mark.parametrize("d,wrap", [(3, 0), (2, 1)])
def test_pair_weight_tables_equal_recomputed_weights(B, d, wrap):
    """The quadratic and reducible pair sums from the weight tables formed once and from weights
    recomputed at every evaluation: the same weights, summed in a different order."""
    N = 8 if d == 3 else 16
    f = _f(d, N, 19)
    kw = dict(M1=4, M2=4) if d == 3 else dict(M=2 * N)
    for precision, tol in (("fp64", 1e-13), ("mixed", 1e-6)):
        a = _gpu_modes(B, d, N, -1.0, f, precision, wrap=wrap, **kw)
        b = _gpu_modes(B, d, N, -1.0, f, precision, wrap=wrap, pair_weights=1, **kw)
        assert np.abs(a - b).max() <= tol * np.abs(a).max()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 1e-6)])
def test_3d_shards_add_up_to_the_evaluation(B, precision, tol):
    """One evaluation split over three shard solvers (as over three GPUs): each returns the modes of
    its output planes (bn_plan_shards) and zero elsewhere; their sum, the one all-reduce of a sharded
    stage, is the unsharded result (the sweep items of a plane are summed by other CTAs, hence the
    tolerance of the precision)."""
    N, eps, count = 12, -1.0, 3
    f = _f(3, N, 23)
    full = _gpu_modes(B, 3, N, eps, f, precision, M1=4, M2=4)
    bounds = B.plan_shards(3, N, count)
    total = np.zeros_like(full)
    for r in range(count):
        part = _gpu_modes(B, 3, N, eps, f, precision, M1=4, M2=4, shard_index=r, shard_count=count)
        outside = np.ones(N, bool)
        outside[bounds[r]:bounds[r + 1]] = False
        assert np.all(part[outside] == 0)
        total += part
    assert np.abs(total - full).max() <= tol * np.abs(full).max()
    prec = B.MIXED if precision == "mixed" else B.FP64
    with B.Solver(3, N, T6, R6, B.HARD_SPHERE, eps, precision=prec, M1=4, M2=4, shard_index=0, shard_count=2) as s:
        s.set_state(f)
        with pytest.raises(B.BNError) as ei:
            s.step_rk(0.01, 1)
        assert ei.value.status == -8


def test_3d_escalation_rebuilds_the_plan(B):
    N, eps, dt = 8, 1.0, 0.01
    f = _f(3, N, 17)
    with B.Solver(3, N, T6, R6, B.HARD_SPHERE, eps, precision=B.MIXED, M1=4, M2=4, escalate_at=1e-9) as s, \
            B.Solver(3, N, T6, R6, B.HARD_SPHERE, eps, precision=B.FP64, M1=4, M2=4) as r:
        s.set_state(f)
        s.step_rk(dt, 1)
        assert s.precision_state()[0] == B.FP64
        r.set_state(s.get_state())
        qa = s.eval_collision_modes()
        qb = r.eval_collision_modes()
    assert np.abs(qa - qb).max() <= 1e-12 * np.abs(qb).max()
