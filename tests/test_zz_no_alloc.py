"""The no-allocation evaluation (include/bn.h: bn_eval_collision_noalloc).

Some callers cannot allocate device memory while they evaluate the operator: cudaMalloc and
cudaFree synchronise the whole device, and they fail when another allocator in the process (a
framework's caching allocator, say) has already reserved the memory.  For them the library offers an
evaluation whose working memory is a fixed file-scope device array instead of solver buffers.  This
test checks, through the C ABI, that it gives the same Q as the ordinary device evaluation
(bn_eval_collision_device) within the tolerances of the other GPU tests, on two calls in a row with
different data (the shared array keeps the previous call's contents), and that a call leaves the
device's free memory unchanged (checked on the second call of each case: the first call in a process
looks up the array's address, which is when the CUDA driver loads the array itself).  The file is collected last so that a failure here comes after every
other test has run.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2110_13735_gb300 import inputs as I

pytestmark = pytest.mark.gpu

R6 = 6.0
T6 = I.box_half_width(R6)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_13735_gb300 import build as BUILD
    BUILD.build()
    from paper_2110_13735_gb300 import bn
    bn.load()
    return torch, bn


CASES = [(32, 1.0, "mixed", 2e-6), (16, -1.0, "fp64", 1e-12), (64, 1.0, "mixed", 2e-6), (24, 0.0, "fp64", 1e-12)]


@pytest.mark.parametrize("N,eps,precision,tol", CASES)
def test_noalloc_matches_device_evaluation(env, N, eps, precision, tol):
    torch, bn = env
    prec = bn.MIXED if precision == "mixed" else bn.FP64
    stream = torch.cuda.current_stream()
    with bn.Solver(2, N, T6, R6, bn.MAXWELL, eps, precision=prec) as s:
        for call in range(2):
            f = I.two_gaussians(2, N, T6, 0.8 + 0.3 * call, (1.5 - call, 0.5 + call), 0.7 - 0.2 * call)
            f_dev = torch.tensor(f.reshape(-1), dtype=torch.float64, device="cuda")
            q_ref = torch.empty_like(f_dev)
            q_na = torch.full_like(f_dev, float("nan"))
            torch.cuda.synchronize()
            s.eval_collision_device(f_dev, q_ref)
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            s.eval_collision_noalloc(f_dev, q_na, stream=stream)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            a, b = q_na.cpu().numpy(), q_ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            err = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert err <= tol, (call, err)
            if call == 1:
                assert free_after == free_before


def test_noalloc_rejects_3d(env):
    torch, bn = env
    with bn.Solver(3, 4, T6, R6, bn.HARD_SPHERE, 1.0, M1=4, M2=4) as s:
        f_dev = torch.ones(64, dtype=torch.float64, device="cuda")
        q = torch.empty_like(f_dev)
        with pytest.raises(bn.BNError) as ei:
            s.eval_collision_noalloc(f_dev, q)
        assert ei.value.status == -8
