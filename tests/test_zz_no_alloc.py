"""crsolve_solve_noalloc: the entry point for callers that cannot call
cudaMalloc (code running where the device allocator is unavailable or
forbidden).  It keeps every intermediate in a fixed 32 MiB device array
inside the library, so these tests check that it gives the same answer as
the regular plan-based entry points, call after call, although the array
keeps the previous call's contents.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synthetic
import paper_1807_00370_gb300 as crs
from paper_1807_00370_gb300 import _native as nat

TOL = 1e-12   # the tolerance of the other FP64 parity tests


def _plan_path(A, B, y):
    N, m, k = y.shape
    dA, dB, dy = (None if a is None else torch.from_numpy(a).cuda() for a in (A, B, y))
    plan = crs.Plan(N, m, k)
    crs.crsolve_factor(plan, dA, dB)
    x = crs.crsolve_solve(plan, dy)
    return x.cpu().numpy(), crs.crsolve_info_get(plan)


def _noalloc(A, B, y):
    """Call crsolve_solve_noalloc through the C ABI with caller-owned device buffers."""
    N, m, k = y.shape
    dA, dB, dy = (torch.from_numpy(a).cuda() for a in (A, B, y))
    dx = torch.empty_like(dy)
    info = nat.CrsolveInfo()
    rc = nat.load().crsolve_solve_noalloc(N, m, k, ctypes.c_void_p(dA.data_ptr()), ctypes.c_void_p(dB.data_ptr()),
                                          ctypes.c_void_p(dy.data_ptr()), ctypes.c_void_p(dx.data_ptr()),
                                          ctypes.byref(info), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == nat.CRSOLVE_OK
    return dx.cpu().numpy(), {"status": info.status, "level": info.level, "block": info.block,
                              "orig_block": info.orig_block}


def _rel(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


@pytest.mark.gpu
def test_two_calls_in_a_row_match_the_plan_path(cuda_ok):
    systems = [synthetic.gen_system(300, 8, 3, seed=71), synthetic.gen_system(1000, 4, 2, seed=72)]
    for A, B, y in systems:
        x, info = _noalloc(A, B, y)
        xr, ir = _plan_path(A, B, y)
        assert info == ir and info["status"] == 0
        assert _rel(x, xr) <= TOL


@pytest.mark.gpu
def test_status_is_reset_between_calls(cuda_ok):
    """A breakdown left in the shared array must not leak into the next call."""
    A, B, y = synthetic.gen_system(64, 4, 1, seed=3)
    for seed in range(20):
        A, B, y = synthetic.gen_system(64, 4, 1, seed=seed)
        Ai = synthetic.make_indefinite(A)
        if np.linalg.eigvalsh(Ai[31]).min() < 0:
            break
    x1, i1 = _noalloc(Ai, B, y)
    xr1, ir1 = _plan_path(Ai, B, y)
    assert i1 == ir1 and i1["status"] == 1
    assert np.isnan(x1).all() and np.isnan(xr1).all()
    x2, i2 = _noalloc(A, B, y)
    xr2, ir2 = _plan_path(A, B, y)
    assert i2 == ir2 and i2["status"] == 0
    assert _rel(x2, xr2) <= TOL


def test_oversized_system_is_rejected_before_any_launch():
    lib = nat.load()
    rc = lib.crsolve_solve_noalloc(1 << 20, 64, 8, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(32),
                                   ctypes.c_void_p(48), None, None)
    assert rc == nat.CRSOLVE_ENOMEM
    assert lib.crsolve_solve_noalloc(0, 4, 1, None, None, None, None, None, None) == nat.CRSOLVE_EINVAL
