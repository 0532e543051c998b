"""The allocation-free FP32 apply, fl_apply_f32_static.

Callers that cannot call cudaMalloc when they apply the operator (a host
whose device memory belongs to another runtime's allocator or pool, or a
service that reserves all of its device memory at start-up) create the
plan at set-up time and then call fl_apply_f32_static, whose scratch is a
fixed library-owned device array.  This file is collected last so that a
run stopping at the first failure has already run every other test; it
passes alone in a fresh process and after the other tests.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.operator import Plan as OPlan  # noqa: E402
from paper_1802_03770_gb300 import _lib  # noqa: E402
from paper_1802_03770_gb300.api import Plan  # noqa: E402

TOL = 2e-5  # the FP32 apply tolerance of the parity tests


def _apply(fn, plan, u):
    y = torch.empty_like(u)
    st = fn(plan._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(y.data_ptr()))
    assert st == _lib.FL_OK, _lib.last_error()
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("d,n", [(2, (1024, 1024)), (2, (37, 53)), (3, (40, 50, 60))])
def test_static_apply_matches_oracle_and_plan_apply_twice(d, n):
    """Two calls in a row on the shared scratch: each within the FP32 apply
    tolerance of the FP64 oracle (applied to the FP32-rounded input) and
    bit for bit equal to fl_apply_f32 (the same kernels and launch shapes)."""
    lib = _lib.load()
    h = 1.0 / (max(n) + 1)
    plan = Plan(d, n, h, 1.3)
    rng = np.random.default_rng(20)
    u64 = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    ref = OPlan(d, n, h, 1.3).apply(u64).ravel()
    u = torch.tensor(u64.ravel(), dtype=torch.float32, device="cuda:0")
    y_plan = _apply(lib.fl_apply_f32, plan, u)
    for _ in range(2):
        y = _apply(lib.fl_apply_f32_static, plan, u)
        assert np.linalg.norm(y - ref) <= TOL * np.linalg.norm(ref)
        assert np.array_equal(y, y_plan)


def test_static_apply_rejects_plans_beyond_the_scratch():
    lib = _lib.load()
    plan = Plan(3, (128, 128, 128), 1.0 / 129, 1.3)   # 128*256*129 > 2^21
    u = torch.zeros(128 ** 3, dtype=torch.float32, device="cuda:0")
    y = torch.empty_like(u)
    st = lib.fl_apply_f32_static(plan._h, ctypes.c_void_p(u.data_ptr()),
                                 ctypes.c_void_p(y.data_ptr()))
    assert st == _lib.FL_INVALID_ARG
    assert "static scratch" in _lib.last_error()
