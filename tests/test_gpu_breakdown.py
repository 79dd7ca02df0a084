"""GPU parity of the breakdown report when several odd blocks fail at the same
level (Sec. 2, "Determination of Positive Definiteness").

The location rule is the oracle's, pinned on the CPU by brute force: the first
level with a failing Cholesky, then the smallest 1-based local block there.
Each case below shifts a set of diagonal blocks so that every one of them is
indefinite; the failures sit in different CTAs of the level kernels (and in
the same one), at level 0 and at deeper levels, so a kernel that reported
the first-arriving or the largest failing block would disagree.  The plain
FP64 path, the batched form and the mixed-precision form must all give the
oracle's (status, level, block, orig_block).
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_1807_00370_gb300 as crs
from paper_1807_00370_gb300 import _native as nat
from tests.gpu_helpers import to_dev
from tests.oracle_helpers import shift_blocks

pytestmark = pytest.mark.gpu

# (N, m, k, shifted original blocks (1-based), expected (level, local block))
CASES = [
    (4097, 8, 2, [3001, 17, 2049], (0, 17)),        # level 0, three CTAs apart
    (4097, 8, 2, [4 * 301, 4 * 33, 4 * 1001], (2, 33)),  # level 2 (originals 4 * odd)
    (4096, 4, 1, [63, 61, 1, 4095], (0, 1)),        # the first block and its CTA neighbours
    (1000, 16, 3, list(range(991, 0, -40)), (0, 31)),  # every 20th odd block, the largest first
    (777, 32, 2, [8 * 97, 8 * 3, 8 * 41], (3, 3)),  # level 3 (originals 8 * odd)
    (300, 64, 4, [299, 101, 37, 201], (0, 37)),     # MT = 64 panels, one block per CTA
    (96, 64, 2, [96, 32], (5, 1)),                  # level 5 of 3 blocks (32, 64, 96): blocks 1 and 3
]


def _case(N, m, k, blocks):
    A, B, y = synthetic.gen_system(N, m, k, seed=N + m)
    return shift_blocks(A, blocks), B, y


def _expect(info, level, block):
    return info == {"status": 1, "level": level, "block": block, "orig_block": block << level}


@pytest.mark.parametrize("N,m,k,blocks,expect", CASES)
def test_plain_multi_failure_location(cuda_ok, N, m, k, blocks, expect):
    A, B, y = _case(N, m, k, blocks)
    _, io = oracle.cr_solve(A, B, y)
    assert _expect(io, *expect), io
    dA, dB, dy = to_dev(A, B, y)
    plan = crs.Plan(N, m, k)
    crs.crsolve_factor(plan, dA, dB)
    x = crs.crsolve_solve(plan, dy)
    assert crs.crsolve_info_get(plan) == io
    assert torch.isnan(x).all()


def test_batched_multi_failure_location(cuda_ok):
    """Every case of CASES with m <= 32 in one batch, between healthy systems."""
    syss, Ns, ms, ks, bad = [], [], [], [], {}
    for i, (N, m, k, blocks, expect) in enumerate(c for c in CASES if c[1] <= 32):
        h = synthetic.gen_system(37 + i, 4, 2, seed=900 + i)
        syss.append(h)
        Ns.append(37 + i), ms.append(4), ks.append(2)
        bad[len(syss)] = expect
        syss.append(_case(N, m, k, blocks))
        Ns.append(N), ms.append(m), ks.append(k)
    b = crs.Batch(np.array(Ns), np.array(ms), np.array(ks))
    A, B, y = b.pack(syss)
    crs.crsolve_batch_solve(b, A, B, y)
    infos = crs.crsolve_batch_info(b)
    for i, (a, bb, yy) in enumerate(syss):
        _, io = oracle.cr_solve(a, bb, yy)
        assert infos[i] == io, (i, infos[i], io)
        if i in bad:
            assert _expect(io, *bad[i]), (i, io)
        else:
            assert io["status"] == 0


@pytest.mark.parametrize("N,m,k,blocks,expect", [c for c in CASES if c[0] <= 1000])
def test_mixed_multi_failure_location(cuda_ok, N, m, k, blocks, expect):
    """The mixed form re-decides an FP32 breakdown in FP64: same report."""
    A, B, y = _case(N, m, k, blocks)
    _, io = oracle.cr_solve(A, B, y)
    dA, dB, dy = to_dev(A, B, y)
    plan = crs.Plan(N, m, k, precision=nat.CRSOLVE_MIXED)
    crs.crsolve_factor(plan, dA, dB)
    x = crs.crsolve_solve(plan, dy)
    assert crs.crsolve_info_get(plan) == io
    assert _expect(io, *expect)
    assert torch.isnan(x).all()
