"""crsolve_solve_noalloc: the entry point for callers that cannot call
cudaMalloc (code running where the device allocator is unavailable or
forbidden, such as a host callback, a pre-allocated real-time loop, or a
plugin that must not grow the device footprint after start-up).  It keeps
every intermediate in a fixed 32 MiB device array inside the library, so
these tests check that its answer equals the oracle's and the regular
plan-based entry points', call after call, although the array keeps the
previous call's contents; that systems one block too large are rejected;
and that a call allocates no device memory.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_1807_00370_gb300 as crs
from paper_1807_00370_gb300 import _native as nat

TOL = 1e-12   # the tolerance of the other FP64 parity tests
ARRAY_BYTES = 32 << 20


def _noalloc_bytes(N, m, k):
    """Bytes of the fixed array that a system needs: the layout the entry
    point documents (per level the odd blocks' factors and right-hand sides,
    the next level's system and vectors, then the CTA-boundary buffers; every
    piece rounded up to 256 bytes)."""
    def up(b):
        return (b + 255) & ~255
    z, cur, Nl = 16, 256, N
    while True:
        no, ne = (Nl + 1) // 2, Nl // 2
        cur += up(no * m * m * z) + up(no * m * 8) + up(no * 2 * m * m * z) + up(no * m * k * z)
        cur += up(ne * m * m * z) + up(max(ne - 1, 0) * m * m * z) + 2 * up(ne * m * k * z)
        if Nl == 1:
            break
        Nl //= 2
    no0 = (N + 1) // 2
    return cur + up(no0 * m * m * z) + up(no0 * m * k * z)


def _largest_fitting_n(m, k):
    lo, hi = 1, ARRAY_BYTES // (m * m * 16) + 1
    while lo + 1 < hi:
        mid = (lo + hi) // 2
        if _noalloc_bytes(mid, m, k) <= ARRAY_BYTES:
            lo = mid
        else:
            hi = mid
    return lo


def _plan_path(A, B, y):
    N, m, k = y.shape
    dA, dB, dy = (None if a is None else torch.from_numpy(a).cuda() for a in (A, B, y))
    plan = crs.Plan(N, m, k)
    crs.crsolve_factor(plan, dA, dB if N > 1 else None)
    x = crs.crsolve_solve(plan, dy)
    return x.cpu().numpy(), crs.crsolve_info_get(plan)


def _c_call(dA, dB, dy, dx, info=None):
    N, m, k = dy.shape
    return nat.load().crsolve_solve_noalloc(
        N, m, k, ctypes.c_void_p(dA.data_ptr()), None if dB is None else ctypes.c_void_p(dB.data_ptr()),
        ctypes.c_void_p(dy.data_ptr()), ctypes.c_void_p(dx.data_ptr()),
        None if info is None else ctypes.byref(info), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _noalloc(A, B, y):
    """Call crsolve_solve_noalloc through the C ABI with caller-owned device
    buffers (B = NULL when N = 1)."""
    N = y.shape[0]
    dA, dy = (torch.from_numpy(a).cuda() for a in (A, y))
    dB = torch.from_numpy(B).cuda() if N > 1 else None
    dx = torch.empty_like(dy)
    info = nat.CrsolveInfo()
    assert _c_call(dA, dB, dy, dx, info) == nat.CRSOLVE_OK
    return dx.cpu().numpy(), {"status": info.status, "level": info.level, "block": info.block,
                              "orig_block": info.orig_block}


def _rel(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


@pytest.mark.gpu
def test_two_calls_in_a_row_match_the_oracle_and_the_plan_path(cuda_ok):
    systems = [synthetic.gen_system(300, 8, 3, seed=71), synthetic.gen_system(1000, 4, 2, seed=72)]
    for A, B, y in systems:
        x, info = _noalloc(A, B, y)
        xo, io = oracle.cr_solve(A, B, y)
        xr, ir = _plan_path(A, B, y)
        assert info == io == ir and info["status"] == 0
        assert _rel(x, xo) <= TOL
        assert _rel(x, xr) <= TOL


@pytest.mark.gpu
def test_single_block_without_b(cuda_ok):
    """N = 1: a plain Cholesky solve; B is NULL."""
    A, _, y = synthetic.gen_system(1, 5, 3, seed=7)
    x, info = _noalloc(A, None, y)
    xo, io = oracle.cr_solve(A, np.zeros((0, 5, 5), np.complex128), y)
    assert info == io and info["status"] == 0
    assert _rel(x, xo) <= TOL


@pytest.mark.gpu
@pytest.mark.parametrize("m,k", [(16, 4), (32, 3), (64, 2)])
def test_largest_system_that_fits(cuda_ok, m, k):
    """The panel Cholesky classes (m > 16) and the largest N whose
    intermediates fit in the array: against the oracle; one block more is
    rejected with CRSOLVE_ENOMEM before anything is enqueued."""
    n = _largest_fitting_n(m, k)
    assert _noalloc_bytes(n + 1, m, k) > ARRAY_BYTES
    A, B, y = synthetic.gen_system(n, m, k, seed=n + m)
    x, info = _noalloc(A, B, y)
    xo, io = oracle.cr_solve(A, B, y)
    assert info == io and info["status"] == 0
    assert _rel(x, xo) <= TOL
    A1, B1, y1 = synthetic.gen_system(n + 1, m, k, seed=1)
    dA, dB, dy = (torch.from_numpy(a).cuda() for a in (A1, B1, y1))
    dx = torch.full_like(dy, 7.0)
    torch.cuda.synchronize()
    assert _c_call(dA, dB, dy, dx) == nat.CRSOLVE_ENOMEM
    torch.cuda.synchronize()
    assert bool((dx == 7.0).all())


@pytest.mark.gpu
def test_status_is_reset_between_calls(cuda_ok):
    """A breakdown left in the shared array must not leak into the next call."""
    for seed in range(20):
        A, B, y = synthetic.gen_system(64, 4, 1, seed=seed)
        Ai = synthetic.make_indefinite(A)
        if np.linalg.eigvalsh(Ai[31]).min() < 0:
            break
    x1, i1 = _noalloc(Ai, B, y)
    _, io1 = oracle.cr_solve(Ai, B, y)
    assert i1 == io1 and i1["status"] == 1
    assert np.isnan(x1).all()
    x2, i2 = _noalloc(A, B, y)
    xo2, io2 = oracle.cr_solve(A, B, y)
    assert i2 == io2 and i2["status"] == 0
    assert _rel(x2, xo2) <= TOL


@pytest.mark.gpu
def test_a_call_allocates_no_device_memory(cuda_ok):
    """Free device memory is the same before and after a call (after a first
    call that loads the kernels)."""
    A, B, y = synthetic.gen_system(500, 8, 4, seed=5)
    dA, dB, dy = (torch.from_numpy(a).cuda() for a in (A, B, y))
    dx = torch.empty_like(dy)
    assert _c_call(dA, dB, dy, dx) == nat.CRSOLVE_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _c_call(dA, dB, dy, dx) == nat.CRSOLVE_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


@pytest.mark.gpu
def test_python_wrapper(cuda_ok):
    """crs.crsolve_solve_noalloc: N = 1 with B = None, and want_info=False
    (asynchronous) followed by a stream synchronisation."""
    A, _, y = synthetic.gen_system(1, 6, 2, seed=9)
    x, info = crs.crsolve_solve_noalloc(torch.from_numpy(A).cuda(), None, torch.from_numpy(y).cuda())
    xo, io = oracle.cr_solve(A, np.zeros((0, 6, 6), np.complex128), y)
    assert info == io
    assert _rel(x.cpu().numpy(), xo) <= TOL
    A, B, y = synthetic.gen_system(257, 12, 5, seed=10)
    dA, dB, dy = (torch.from_numpy(a).cuda() for a in (A, B, y))
    x, info = crs.crsolve_solve_noalloc(dA, dB, dy, want_info=False)
    assert info is None
    torch.cuda.current_stream().synchronize()
    xo, _ = oracle.cr_solve(A, B, y)
    assert _rel(x.cpu().numpy(), xo) <= TOL
    xr, _ = _plan_path(A, B, y)
    assert _rel(x.cpu().numpy(), xr) <= TOL


def test_oversized_system_is_rejected_before_any_launch():
    lib = nat.load()
    rc = lib.crsolve_solve_noalloc(1 << 20, 64, 8, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(32),
                                   ctypes.c_void_p(48), None, None)
    assert rc == nat.CRSOLVE_ENOMEM
    # sizes whose byte counts would overflow a 64-bit product
    for n in ((1 << 62) + 1, (1 << 40), (1 << 60)):
        assert lib.crsolve_solve_noalloc(n, 64, 8, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(32),
                                         ctypes.c_void_p(48), None, None) == nat.CRSOLVE_ENOMEM
    assert lib.crsolve_solve_noalloc(0, 4, 1, None, None, None, None, None, None) == nat.CRSOLVE_EINVAL


def test_layout_bound_matches_the_documented_estimate():
    """The documented rule of thumb (about N (5.5 m^2 + 3.5 m k) 16 bytes)
    against the exact layout, and N ~ 4500 for m = 8, k = 4."""
    for m, k in ((4, 1), (8, 4), (16, 8), (64, 32)):
        n = 4096 if m <= 16 else 64
        est = n * (5.5 * m * m + 3.5 * m * k) * 16
        assert 0.9 * est <= _noalloc_bytes(n, m, k) <= 1.15 * est + 64 * 1024, (m, k)
    assert 4300 <= _largest_fitting_n(8, 4) <= 4700
