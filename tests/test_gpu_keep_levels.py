"""Plans split by crsolve_plan_keep_levels: the workspace keeps the factors of
the fine levels 0 .. keep-1 and the level-keep reduced system, the scratch
holds the coarse levels and the solve buffers.  After the scratch is released
and a new one bound, the next solve or backward re-factors the coarse levels
from the stored level-keep system.  That re-factorisation runs the same
kernels on the same inputs, so every result must be bit-identical to an
unsplit plan's; the unsplit results themselves are checked against the CPU
oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_1807_00370_gb300 as crs
from paper_1807_00370_gb300 import _native as nat
from tests.gpu_helpers import rel_err, to_dev

pytestmark = pytest.mark.gpu


def _rebind_elsewhere(plan):
    """Release the scratch and bind a new one at another address; the old
    memory is overwritten (held by a NaN-filled tensor meanwhile), so stale
    coarse factors cannot be read back by accident."""
    plan.release_scratch()
    poison = torch.full((max(plan.scratch_bytes, 256) // 8,), float("nan"), dtype=torch.float64,
                        device=plan.device)
    plan.ensure_scratch()
    torch.cuda.synchronize()
    return poison


@pytest.mark.parametrize("N,m,k", [(1000, 8, 4), (333, 16, 3), (4097, 4, 2), (65, 32, 5), (2, 3, 1)])
def test_split_plans_are_bit_identical(cuda_ok, N, m, k):
    A, B, y = synthetic.gen_system(N, m, k, seed=3 * N + m)
    c = synthetic.gen_cotangent(N, m, k, seed=3 * N + m)
    dA, dB, dy, dc = to_dev(A, B if N > 1 else None, y, c)
    ref = crs.Plan(N, m, k)
    crs.crsolve_factor(ref, dA, dB)
    x_ref = crs.crsolve_solve(ref, dy)
    g_ref = crs.crsolve_backward(ref, x_ref, dc)
    xo, _ = oracle.cr_solve(A, B, y)
    assert rel_err(x_ref, xo) <= 1e-12
    nlev = len(crs.crsolve_plan_levels(ref))
    sizes = []
    for keep in sorted({0, 1, 2, nlev - 1, nlev}):
        plan = crs.Plan(N, m, k, keep_levels=keep)
        # the two regions together are exactly the unsplit workspace
        assert plan.workspace_bytes + plan.scratch_bytes == ref.workspace_bytes
        sizes.append(plan.workspace_bytes)
        crs.crsolve_factor(plan, dA, dB)
        assert torch.equal(crs.crsolve_solve(plan, dy), x_ref), keep
        poison = _rebind_elsewhere(plan)
        assert torch.equal(crs.crsolve_solve(plan, dy), x_ref), keep
        poison = _rebind_elsewhere(plan)
        g = crs.crsolve_backward(plan, x_ref, dc)
        for a, b in zip(g, g_ref):
            assert (a is None and b is None) or torch.equal(a, b), keep
        del poison
    assert sizes == sorted(sizes)


def test_keep_one_level_holds_about_half_the_factors(cuda_ok):
    N, m, k = 1 << 14, 8, 4
    full = crs.Plan(N, m, k, keep_levels=64)
    half = crs.Plan(N, m, k, keep_levels=1)
    none = crs.Plan(N, m, k, keep_levels=0)
    factors = full.workspace_bytes - none.workspace_bytes
    kept = half.workspace_bytes - none.workspace_bytes
    assert 0.45 * factors <= kept <= 0.55 * factors, (kept, factors)


def test_split_plan_breakdown_flags_survive_refactor(cuda_ok):
    N, m = 512, 8
    for seed in range(20):
        A, B, y = synthetic.gen_system(N, m, 2, seed=seed)
        Ai = synthetic.make_indefinite(A)
        if np.linalg.eigvalsh(Ai[N // 2 - 1]).min() < 0:
            break
    _, io = oracle.cr_solve(Ai, B, y)
    assert io["status"] == 1
    dA, dB, dy = to_dev(Ai, B, y)
    for keep in (0, 2, 5):
        plan = crs.Plan(N, m, 2, keep_levels=keep)
        crs.crsolve_factor(plan, dA, dB)
        assert np.isnan(crs.crsolve_solve(plan, dy).cpu().numpy()).all()
        assert crs.crsolve_info_get(plan) == io
        poison = _rebind_elsewhere(plan)
        assert np.isnan(crs.crsolve_solve(plan, dy).cpu().numpy()).all()
        assert crs.crsolve_info_get(plan) == io, keep
        del poison


def test_split_plan_errors(cuda_ok):
    N, m, k = 100, 8, 2
    A, B, y = synthetic.gen_system(N, m, k, seed=5)
    dA, dB, dy = to_dev(A, B, y)
    plan = crs.Plan(N, m, k, keep_levels=2)
    crs.crsolve_factor(plan, dA, dB)
    plan.release_scratch()
    lib = nat.load()
    x = torch.empty_like(dy)
    # no scratch bound: the C ABI refuses before launching anything
    rc = lib.crsolve_solve(plan.handle, k, dy.data_ptr(), x.data_ptr(), None)
    assert rc == nat.CRSOLVE_ENOMEM
    # the split is fixed once memory is bound; unsplit plans have no scratch
    assert lib.crsolve_plan_keep_levels(plan.handle, 1) == nat.CRSOLVE_EINVAL
    ref = crs.Plan(N, m, k)
    assert lib.crsolve_set_scratch(ref.handle, None, 0) == nat.CRSOLVE_EINVAL
    # only classic FP64 plans split
    with pytest.raises(nat.CrsolveError):
        crs.Plan(N, m, k, precision=nat.CRSOLVE_MIXED, keep_levels=1)
    with pytest.raises(nat.CrsolveError):
        crs.Plan(128, m, k, flags=nat.CRSOLVE_PLAN_ALG1, keep_levels=1)


@pytest.mark.parametrize("keep", [False, 1, 3])
def test_autograd_keep_levels_gives_identical_gradients(cuda_ok, keep):
    N, m, k = 2000, 8, 4
    A, B, y = synthetic.gen_system(N, m, k, seed=11)
    c = synthetic.gen_cotangent(N, m, k, seed=11)
    grads = []
    for kf in (True, keep):
        tA, tB, ty = (t.requires_grad_() for t in to_dev(A, B, y))
        x = crs.CRSolveFn.apply(tA, tB, ty, kf)
        loss = (torch.from_numpy(c).cuda().conj() * x).real.sum()
        loss.backward()
        grads.append((tA.grad, tB.grad, ty.grad))
    for a, b in zip(*grads):
        assert torch.equal(a, b)


def test_split_plan_host_buffers(cuda_ok):
    """crsolve_solve_host on a split plan stages A, B, y and x in the scratch;
    x equals the device path.  With keep >= 1 a later device solve after a new
    scratch rebuilds the coarse levels from the kept level-keep system; with
    keep = 0 the staged level-0 system is gone with the scratch, so that solve
    is refused (CRSOLVE_ENOTFACTORED) instead of reading lost data."""
    N, m, k = 3000, 8, 4
    A, B, y = synthetic.gen_system(N, m, k, seed=21)
    dA, dB, dy = to_dev(A, B, y)
    ref = crs.Plan(N, m, k)
    crs.crsolve_factor(ref, dA, dB)
    x_ref = crs.crsolve_solve(ref, dy)
    tA, tB, ty = (torch.from_numpy(a).pin_memory() for a in (A, B, y))
    for keep in (0, 1, 3):
        plan = crs.Plan(N, m, k, flags=nat.CRSOLVE_PLAN_HOST_STAGING, keep_levels=keep)
        x, rc = crs.crsolve_solve_host(plan, tA, tB, ty)
        assert rc == 0 and torch.equal(x, x_ref.cpu()), keep
        poison = _rebind_elsewhere(plan)
        if keep == 0:
            with pytest.raises(nat.CrsolveError):
                crs.crsolve_solve(plan, dy)
        else:
            assert torch.equal(crs.crsolve_solve(plan, dy), x_ref), keep
        del poison


def test_mixed_plan_after_host_solve_uses_its_fp64_factors(cuda_ok):
    """A mixed plan factored by crsolve_factor on one system and then used by
    crsolve_solve_host on another: a later crsolve_solve must solve the second
    system (the host path's FP64 factors), not refine with the first one's."""
    N, m, k = 500, 8, 2
    A1, B1, y1 = synthetic.gen_system(N, m, k, seed=31)
    A2, B2, y2 = synthetic.gen_system(N, m, k, seed=32)
    d1 = to_dev(A1, B1, y1)
    plan = crs.Plan(N, m, k, precision=nat.CRSOLVE_MIXED, flags=nat.CRSOLVE_PLAN_HOST_STAGING)
    crs.crsolve_factor(plan, d1[0], d1[1])
    x2h, rc = crs.crsolve_solve_host(plan, *(torch.from_numpy(a).pin_memory() for a in (A2, B2, y2)))
    assert rc == 0
    xo2, _ = oracle.cr_solve(A2, B2, y2)
    assert rel_err(x2h.numpy(), xo2) <= 1e-12
    (dy2,) = to_dev(y2)
    assert rel_err(crs.crsolve_solve(plan, dy2), xo2) <= 1e-12
