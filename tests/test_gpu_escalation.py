"""Precision escalation: a mixed-precision solver switches to FP64 for good once |eps| max f reaches
its threshold (near Fermi saturation f -> 1/|eps| or at the onset of Bose condensation), and every
step after the switch agrees with the FP64 oracle to FP64 tolerance, alone and inside a batch."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2110_13735_gb300 import inputs as I

pytestmark = pytest.mark.gpu

R6 = 6.0
T6 = I.box_half_width(R6)
N, DT = 16, 0.005


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


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _boson_f0():
    return I.gaussian(2, N, T6, 5.0, 0.5)   # max f0 = 5 / pi > 1


def test_escalates_once_and_then_matches_fp64(B):
    f0 = _boson_f0()
    ora = O.Operator(2, N, T6, R6, 0, 1.0, M=2 * N)
    with B.Solver(2, N, T6, R6, B.MAXWELL, 1.0, precision=B.MIXED, escalate_at=1.0) as s:
        s.set_state(f0)
        assert s.precision_state() == (B.MIXED, -1.0, 0.0)
        s.step_rk(DT, 1)
        f1 = s.get_state()
        p, t_esc, mf = s.precision_state()
        assert p == B.FP64
        assert t_esc == pytest.approx(DT, rel=1e-15)
        assert mf == float(f1.max())
        # the first step ran in mixed precision
        assert 1e-12 < rel(f1, ora.step(f0, DT, 1, 0)) < 1e-5
        s.step_rk(DT, 3)
        f4 = s.get_state()
        assert s.precision_state()[:2] == (B.FP64, pytest.approx(DT, rel=1e-15))
    assert rel(f4, ora.step(f1, DT, 3, 0)) <= 1e-12


def test_below_threshold_stays_mixed(B):
    f0 = _boson_f0()
    kw = dict(precision=B.MIXED, escalate_at=50.0)
    with B.Solver(2, N, T6, R6, B.MAXWELL, 1.0, **kw) as s, B.Solver(2, N, T6, R6, B.MAXWELL, 1.0, **kw) as one:
        s.set_state(f0)
        one.set_state(f0)
        s.step_rk(DT, 3)
        p, t_esc, mf = s.precision_state()
        maxima = []
        for _ in range(3):
            one.step_rk(DT, 1)
            maxima.append(float(one.get_state().max()))
            assert one.precision_state()[2] == maxima[-1]
        assert np.array_equal(s.get_state(), one.get_state())
    assert (p, t_esc) == (B.MIXED, -1.0)
    # the monitor reports the largest f seen at the end of any step of the call
    assert mf == max(maxima)


def test_classical_never_escalates(B):
    # eps = 0: |eps| max f = 0 whatever f is
    f0 = _boson_f0()
    with B.Solver(2, N, T6, R6, B.MAXWELL, 0.0, precision=B.MIXED, escalate_at=1e-9) as s:
        s.set_state(f0)
        s.step_rk(DT, 2)
        assert s.precision_state()[:2] == (B.MIXED, -1.0)


def test_escalation_inside_a_batch(B):
    f0 = _boson_f0()
    g0 = I.two_gaussians(2, 32, T6, 1.0, (2.0, 1.0), 0.8)
    ora = O.Operator(2, N, T6, R6, 0, 1.0, M=2 * N)
    with B.Solver(2, N, T6, R6, B.MAXWELL, 1.0, precision=B.MIXED, escalate_at=1.0) as a, \
            B.Solver(2, 32, T6, R6, B.MAXWELL, -1.0, precision=B.MIXED, escalate_at=0.95) as b, \
            B.Solver(2, 32, T6, R6, B.MAXWELL, -1.0, precision=B.MIXED) as alone:
        a.set_state(f0)
        b.set_state(g0)
        alone.set_state(g0)
        assert B.step_rk_batch([a, b], [DT, 0.01], 1) == -1
        assert a.precision_state()[0] == B.FP64
        assert b.precision_state()[0] == B.MIXED      # max f = 0.8 < 0.95
        f1 = a.get_state()
        # the batch is rebuilt without the escalated solver's mixed plan
        assert B.step_rk_batch([a, b], [DT, 0.01], 2) == -1
        alone.step_rk(0.01, 3)
        assert rel(a.get_state(), ora.step(f1, DT, 2, 0)) <= 1e-12
        assert np.array_equal(b.get_state(), alone.get_state())
