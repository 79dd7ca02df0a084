"""GPU parity of the CTA-boundary completion inside the odd-block kernels of
the plain path (the second of the two CTAs beside a chunk boundary completes
its even block; no fix-up launch; used for launches of at most four CTAs per
SM, the finer levels keep the fix-up kernel): x equals the oracle's within
the FP64 tolerance and, bit for bit, the batched form's (whose single CTA per
system completes the boundaries in chunk order) and the host-buffer path's
(whose level-0 factor wavefront keeps the fix-up kernels), on levels of
hundreds of CTAs, several right-hand-side column chunks (level 0 of the
k = 17 and k = 9 cases takes the fix-up kernel, the levels below do not) and
a ragged last chunk, call after call."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_1807_00370_gb300 as crs
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.mark.parametrize("N,m,k", [(16411, 4, 1), (16411, 8, 17), (9001, 16, 9), (5003, 5, 3)])
def test_fused_boundaries_match_oracle_batched_and_fixup_paths(cuda_ok, N, m, k):
    A, B, y = synthetic.gen_system(N, m, k, seed=N + m + k)
    dA, dB, dy = (torch.from_numpy(a).cuda() for a in (A, B, y))
    plan = crs.Plan(N, m, k, flags=1)   # host staging too, for the host-buffer path
    xs = []
    for _ in range(3):   # the arrival counters are reused call after call
        crs.crsolve_factor(plan, dA, dB)
        xs.append(crs.crsolve_solve(plan, dy).cpu().numpy())
    assert all(np.array_equal(xs[0], x) for x in xs[1:])
    xo, io = oracle.cr_solve(A, B, y)
    assert crs.crsolve_info_get(plan) == io and io["status"] == 0
    assert rel_err(xs[0], xo) <= TOL
    # host buffers: the level-0 factor and the wavefront keep the fix-up kernels
    tA, tB, ty = (torch.from_numpy(a).pin_memory() for a in (A, B, y))
    tx = torch.empty_like(ty).pin_memory()
    crs.crsolve_solve_host(plan, tA, tB, ty, tx)
    assert np.array_equal(tx.numpy(), xs[0])
    b = crs.Batch([N], [m], [k])
    bA, bB, by = b.pack([(A, B, y)])
    xb = crs.crsolve_batch_solve(b, bA, bB, by)
    assert np.array_equal(b.system_view(0, bA, bB, xb)[2].cpu().numpy(), xs[0])


def test_one_launch_per_factor_level(cuda_ok):
    """At N = 2^13, m = 8 every level has at most 256 CTAs: the factor issues
    one kernel per level (and a memset), the solve one per level and sweep,
    no fix-up launches."""
    N, m, k = 1 << 13, 8, 4
    A, B, y = synthetic.gen_system(N, m, k, seed=3)
    dA, dB, dy = (torch.from_numpy(a).cuda() for a in (A, B, y))
    plan = crs.Plan(N, m, k)
    nlev = N.bit_length()   # levels of 2^13, 2^12, ..., 1 blocks
    c0 = crs.crsolve_launch_count(plan)
    crs.crsolve_factor(plan, dA, dB)
    c1 = crs.crsolve_launch_count(plan)
    x = crs.crsolve_solve(plan, dy)
    c2 = crs.crsolve_launch_count(plan)
    assert c1 - c0 == nlev
    assert c2 - c1 == 2 * nlev
    xo, _ = oracle.cr_solve(A, B, y)
    assert rel_err(x.cpu().numpy(), xo) <= TOL
