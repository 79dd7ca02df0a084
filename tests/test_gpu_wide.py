"""GPU parity of the wide forms of the block classes m <= 16 (right-looking
Cholesky and substitutions by (block, row, column) items), which the plain
path runs on its coarse levels: x equals the oracle's within the FP64
tolerance and, bit for bit, the batched form's, which runs the same levels
with a column per thread.  The sizes put levels at one, two and four odd
blocks per CTA and at narrowed right-hand-side chunks, with ragged m and k."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_1807_00370_gb300 as crs
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _plain(A, B, y):
    N, m, k = y.shape
    plan = crs.Plan(N, m, k)
    crs.crsolve_factor(plan, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda() if N > 1 else None)
    return crs.crsolve_solve(plan, torch.from_numpy(y).cuda()).cpu().numpy(), crs.crsolve_info_get(plan)


def _batched(systems):
    Ns = [s[2].shape[0] for s in systems]
    ms = [s[2].shape[1] for s in systems]
    ks = [s[2].shape[2] for s in systems]
    b = crs.Batch(Ns, ms, ks)
    A, B, y = b.pack(systems)
    x = crs.crsolve_batch_solve(b, A, B, y)
    infos = crs.crsolve_batch_info(b)
    return [b.system_view(i, A, B, x)[2].cpu().numpy() for i in range(len(systems))], infos


@pytest.mark.parametrize("m,k", [(1, 1), (3, 5), (4, 8), (5, 2), (8, 4), (8, 17), (11, 3), (16, 8), (16, 1)])
def test_wide_levels_match_oracle_and_column_per_thread_form(cuda_ok, m, k):
    # N = 2500: level 0 has 1250 odd blocks, so the levels below run at four,
    # two and one odd blocks per CTA (about two CTAs per SM)
    systems = [synthetic.gen_system(N, m, k, seed=900 + 10 * m + k) for N in (2500, 611, 40)]
    xb, ib = _batched(systems)
    for i, (A, B, y) in enumerate(systems):
        xp, ip = _plain(A, B, y)
        xo, io = oracle.cr_solve(A, B, y)
        assert ip == io == ib[i] and io["status"] == 0
        assert rel_err(xp, xo) <= TOL, (i, rel_err(xp, xo))
        assert np.array_equal(xp, xb[i]), f"N={y.shape[0]}, m={m}, k={k}: wide and column-per-thread forms differ"


@pytest.mark.parametrize("m", [4, 16])
def test_breakdown_on_a_wide_level(cuda_ok, m):
    """A_{N/2} - 3I first fails on a coarse level (level log2(N/2) for N a
    power of two), whose factor runs the right-looking Cholesky: the same
    flags and location as the oracle, x all NaN."""
    N = 512
    for seed in range(40):
        A, B, y = synthetic.gen_system(N, m, 2, seed=seed)
        Ai = synthetic.make_indefinite(A)
        _, io = oracle.cr_solve(Ai, B, y)
        if io["status"] == 1 and io["level"] >= 4:
            break
    else:
        pytest.skip("no seed gave a coarse-level breakdown")
    xp, ip = _plain(Ai, B, y)
    assert ip == io
    assert np.isnan(xp).all()
    xb, ib = _batched([(Ai, B, y)])
    assert ib[0] == io
