"""The bounded-wait error path of the operator kernels, exercised without any fault.

Every wait of a kernel for a bulk (TMA) copy is bounded; when it runs out the kernel records it,
waits (bounded) for its copy before going on or returning, and the call returns BN_ERR_TIMEOUT.
The testing option debug_wait_giveup makes the first wait of each operator kernel give up at once,
so the path runs on every call of such a solver.  The test checks the status, that
the context stays usable (an ordinary solver evaluates correctly right after), and that the flag
does not stick to later calls of that ordinary solver.
"""
from __future__ import annotations

import numpy as np
import pytest

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


CASES = [(2, 16, "mixed"), (2, 16, "fp64"), (2, 64, "mixed"), (3, 8, "mixed"), (3, 8, "fp64")]


@pytest.mark.parametrize("d,N,precision", CASES)
def test_wait_runs_out_and_the_context_survives(B, d, N, precision):
    prec = B.MIXED if precision == "mixed" else B.FP64
    kernel = B.HARD_SPHERE if d == 3 else B.MAXWELL
    kw = dict(M1=4, M2=4) if d == 3 else {}
    f = I.two_gaussians(d, N, T6, 1.0, (1.5, 0.0, 0.0)[:d] if d == 3 else (1.5, 0.5), 0.8)
    with B.Solver(d, N, T6, R6, kernel, 1.0, precision=prec, debug_wait_giveup=1, **kw) as s:
        s.set_state(f)
        with pytest.raises(B.BNError) as ei:
            s.eval_collision()
        assert ei.value.status == -6
        with pytest.raises(B.BNError) as ei:
            s.step_rk(0.01, 1)
        assert ei.value.status == -6
    with B.Solver(d, N, T6, R6, kernel, 1.0, precision=prec, **kw) as r1, \
            B.Solver(d, N, T6, R6, kernel, 1.0, precision=prec, **kw) as r2:
        r1.set_state(f)
        r2.set_state(f)
        a = r1.eval_collision()
        b = r2.eval_collision()
        c = r1.eval_collision()
    assert np.all(np.isfinite(a))
    assert np.array_equal(a, b) and np.array_equal(a, c)
