"""Host-side checks of the C-ABI library (no GPU needed): it builds for sm_103a, loads, exports
every function declared in include/bn.h, and validates arguments before touching a device."""
from __future__ import annotations

import ctypes

import pytest

from paper_2110_13735_gb300 import bn as B
from paper_2110_13735_gb300 import build as BUILD


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.load()


def test_exports_every_declared_symbol(lib):
    names = B.declared_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_the_binding(lib):
    """The binding declares bn_options and bn_request itself: their sizes must be the library's."""
    assert lib.bn_options_bytes() == ctypes.sizeof(B.Options)
    assert lib.bn_request_bytes() == ctypes.sizeof(B.Request)


def test_default_options_and_last_error(lib):
    o = B.Options()
    assert lib.bn_default_options(ctypes.byref(o)) == 0
    assert (o.M, o.precision, o.conserve, o.integrator) == (0, 0, 0, 0)
    assert lib.bn_default_options(None) == -1
    assert b"NULL" in lib.bn_last_error()


@pytest.mark.parametrize("args,status", [
    ((1, 16, 13.3, 6.0, 0, 0.0), -1),      # d
    ((2, 15, 13.3, 6.0, 0, 0.0), -1),      # odd N
    ((2, 2, 13.3, 6.0, 0, 0.0), -1),       # N too small
    ((2, 128, 13.3, 6.0, 0, 0.0), -8),     # N too large
    ((2, 16, 13.0, 6.0, 0, 0.0), -2),      # anti-aliasing violated (T < (3+sqrt2) R / 2)
    ((2, 16, -1.0, 6.0, 0, 0.0), -1),      # T
    ((3, 8, 13.3, 6.0, 0, 0.0), -8),       # 3-D Maxwell
    ((2, 16, 13.3, 6.0, 7, 0.0), -1),      # unknown kernel
    ((2, 16, 13.3, 6.0, 0, float("nan")), -1),
])
def test_create_rejects_bad_arguments_without_a_device(lib, args, status):
    h = ctypes.c_void_p()
    st = lib.bn_create_solver(*args, None, None, ctypes.byref(h))
    assert st == status, lib.bn_last_error()
    assert not h.value


def test_create_rejects_bad_escalation_threshold(lib):
    for bad in (-0.5, float("nan"), float("inf")):
        o = B.options(precision=B.MIXED, escalate_at=bad)
        h = ctypes.c_void_p()
        st = lib.bn_create_solver(2, 16, 13.3, 6.0, 0, 1.0, ctypes.byref(o), None, ctypes.byref(h))
        assert st == -1, bad
        assert b"escalate_at" in lib.bn_last_error()
        assert not h.value
    assert lib.bn_precision_state(None, None, None, None) == -1
    o = B.options(precision=B.MIXED, mixed_rw=12)
    h = ctypes.c_void_p()
    assert lib.bn_create_solver(2, 16, 13.3, 6.0, 0, 1.0, ctypes.byref(o), None, ctypes.byref(h)) == -1
    assert b"mixed_rw" in lib.bn_last_error()
    assert lib.bn_kernel_config(None, None, 0) == -1
    o = B.options(precision=B.MIXED, mixed_variant=5)
    assert lib.bn_create_solver(2, 16, 13.3, 6.0, 0, 1.0, ctypes.byref(o), None, ctypes.byref(h)) == -1


def test_null_handles(lib):
    assert lib.bn_set_state(None, None, 0) == -1
    # the no-allocation evaluation checks its arguments before any CUDA call
    assert lib.bn_eval_collision_noalloc(None, None, None, 0, None) == -1
    assert lib.bn_step_rk(None, 0.1, 1) == -1
    assert lib.bn_kernel_launches(None) == 0
    # velocity rescaling: every entry point rejects a null solver before any device work
    assert lib.bn_rescale_set(None, 4.0, 1.0, None, 2, 1.0, 1.0) == -1
    assert lib.bn_step_rescaled(None, 0.1, 1) == -1
    assert lib.bn_step_rescaled_rk2(None, 0.1, 1) == -1
    assert lib.bn_rescale_get(None, None, 9) == -1
    lib.bn_destroy_solver(None)


def test_server_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.bn_server_create(0, 0, None, ctypes.byref(h)) == -1
    assert lib.bn_server_submit(None, None, None, 0, None) == -1
    assert lib.bn_server_poll(None, 1, None, None, 0, None, 0) == -1
    lib.bn_server_destroy(None)
