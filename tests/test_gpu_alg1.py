"""GPU parity of the Algorithm 1 path (plans with CRSOLVE_PLAN_ALG1: the
paper's own recursion, both halves reduced at every level) against the CPU
oracle of Algorithm 1 and, since both methods reach x = A^{-1} y, the
classic oracle.

Tolerances as for the classic path: 1e-12 on the default generator
(kappa <= ~10; both solvers are backward stable with backward error about
c * m * log2(N) * 2^-53), 1e-10 on a kappa ~ 1e6 system.  Breakdown status,
depth and original block must match the oracle exactly; the reported
position is the original block's place among the N blocks of that depth.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_1807_00370_gb300 as crs
from paper_1807_00370_gb300 import _native as nat
from tests.gpu_helpers import rel_err, to_dev
from tests.oracle_helpers import assemble, brute_force_first_failure, herm_from_lower

pytestmark = pytest.mark.gpu

TOL = 1e-12
ALG1 = nat.CRSOLVE_PLAN_ALG1


def run(A, B, y, kmax=None):
    N, m, k = y.shape
    dA, dB, dy = to_dev(A, B if N > 1 else None, y)
    plan = crs.Plan(N, m, kmax or k, flags=ALG1)
    crs.crsolve_factor(plan, dA, dB)
    x = crs.crsolve_solve(plan, dy)
    info = crs.crsolve_info_get(plan)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info, plan


def position(orig, level, N):
    """1-based place of original block `orig` among the N blocks of depth
    `level`: rotr^level of orig - 1 on log2 N bits."""
    L = N.bit_length() - 1
    if L == 0:
        return orig
    s, u, mask = level % L, orig - 1, N - 1
    return (((u >> s) | (u << (L - s))) & mask) + 1 if s else orig


def expect_info(io, N):
    if io["status"] == 0:
        return {"status": 0, "level": 0, "block": 0, "orig_block": 0}
    return {"status": 1, "level": io["level"], "block": position(io["orig_block"], io["level"], N),
            "orig_block": io["orig_block"]}


def test_small_system(cuda_ok):
    A, B, y = synthetic.gen_system(64, 4, 1, seed=0)
    x, info, _ = run(A, B, y)
    xo, io = oracle.alg1_solve(A, B, y)
    assert info == expect_info(io, 64) and info["status"] == 0
    assert rel_err(x, xo) <= TOL


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7, 8, 9, 12, 16, 20, 32, 33, 48, 64])
def test_every_block_size(cuda_ok, m):
    N = 64 if m <= 16 else 16
    A, B, y = synthetic.gen_system(N, m, 3, seed=m)
    x, info, _ = run(A, B, y)
    xo, io = oracle.alg1_solve(A, B, y)
    assert info["status"] == 0 == io["status"]
    assert rel_err(x, xo) <= TOL


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 32, 64, 128, 256, 1024, 4096, 16384])
def test_sizes_span_tiles_and_ragged_tails(cuda_ok, N):
    """Every level runs a reduction of N/2 and one of N/2 + 1 odd blocks, so
    each level has a ragged last chunk."""
    A, B, y = synthetic.gen_system(N, 8, 4, seed=N)
    x, info, _ = run(A, B, y)
    xo, io = oracle.alg1_solve(A, B, y)
    assert info["status"] == 0 == io["status"]
    assert rel_err(x, xo) <= TOL
    xc, _ = oracle.cr_solve(A, B, y)
    assert rel_err(x, xc) <= TOL


@pytest.mark.parametrize("k", [1, 2, 5, 16, 33, 64])
def test_rhs_widths(cuda_ok, k):
    A, B, y = synthetic.gen_system(256, 8, k, seed=50 + k)
    x, info, _ = run(A, B, y, kmax=max(k, 40))
    xo, _ = oracle.alg1_solve(A, B, y)
    assert info["status"] == 0
    assert rel_err(x, xo) <= TOL


def test_levels_of_the_plan(cuda_ok):
    plan = crs.Plan(1024, 4, 1, flags=ALG1)
    assert crs.crsolve_plan_levels(plan) == [1024] * 11


def test_lower_triangle_only_and_real_diagonal(cuda_ok):
    A, B, y = synthetic.gen_system(32, 5, 2, seed=8)
    x, _, _ = run(A, B, y)
    A2 = A.copy()
    iu = np.triu_indices(5, 1)
    A2[:, iu[0], iu[1]] = 1e3 * (1 - 3j)
    A2[:, np.arange(5), np.arange(5)] += 5j
    x2, _, _ = run(A2, B, y)
    assert np.array_equal(x, x2)


def test_breakdown_flags_and_locations_on_random_systems(cuda_ok):
    """Status, first failing depth and smallest failing original block equal
    the oracle's, on random systems made indefinite at chosen blocks (only
    cases whose eigenvalues keep a margin from zero)."""
    rng = np.random.default_rng(77)
    depths, seen = set(), {True: 0, False: 0}
    for trial in range(60):
        N = 1 << int(rng.integers(0, 6))
        m = int(rng.integers(1, 5))
        A, B, y = synthetic.gen_system(N, m, 2, seed=3000 + trial, shift=0.2)
        lam = np.linalg.eigvalsh(assemble(A, B))
        blk = min(np.linalg.eigvalsh(herm_from_lower(a)).min() for a in A)
        A = A.copy()
        r = rng.random()
        if r < 0.4:
            # just below the smallest eigenvalue, every diagonal block still
            # positive definite: the failure surfaces at a deeper split
            A = A - (lam.min() + 10 ** rng.uniform(-3, -0.3) * (blk - lam.min())) * np.eye(m)
        elif r < 0.6:
            A = A - float(rng.uniform(0, 1.2 * lam.max())) * np.eye(m)
        else:
            tau = float(rng.uniform(0, 1.2 * lam.max()))
            for b in rng.choice(N, size=int(rng.integers(1, N + 1)), replace=False):
                A[b] -= float(rng.uniform(0, tau)) * np.eye(m)
        try:
            expect = brute_force_first_failure(A, B, 1e-9 * lam.max())
        except ValueError:
            continue
        x, info, _ = run(A, B, y)
        xo, io = oracle.alg1_solve(A, B, y)
        assert info == expect_info(io, N), (trial, N, m, info, io)
        if expect is not None:
            assert (io["level"], io["orig_block"]) == expect
            assert np.isnan(x).all()
            depths.add(expect[0])
        else:
            assert rel_err(x, xo) <= 1e-11
        seen[expect is not None] += 1
    assert seen[True] >= 8 and seen[False] >= 8 and len(depths) >= 4


def test_indefinite_block_is_found_at_depth_zero(cuda_ok):
    N, m = 4096, 8
    for seed in range(20):
        A, B, y = synthetic.gen_system(N, m, 4, seed=seed)
        Ai = synthetic.make_indefinite(A)
        if np.linalg.eigvalsh(herm_from_lower(Ai[N // 2 - 1])).min() < 0:
            break
    x, info, _ = run(Ai, B, y)
    _, io = oracle.alg1_solve(Ai, B, y)
    assert info == expect_info(io, N) == {"status": 1, "level": 0, "block": N // 2, "orig_block": N // 2}
    assert np.isnan(x).all()


def test_nan_input_reports_breakdown(cuda_ok):
    A, B, y = synthetic.gen_system(16, 3, 1, seed=4)
    A[5, 2, 1] = np.nan
    x, info, _ = run(A, B, y)
    _, io = oracle.alg1_solve(A, B, y)
    assert info == expect_info(io, 16) and info["level"] == 0 and info["orig_block"] == 6
    assert np.isnan(x).all()


def test_kappa_1e6_matches_oracle(cuda_ok):
    path = os.path.join(os.path.dirname(__file__), "golden", "kappa_shifts.json")
    case = json.load(open(path))["plain_N2p12_m8_k4"]
    A, B, y = synthetic.gen_system(case["N"], case["m"], case["k"], seed=case["seed"],
                                   shift=case["shifts"]["1e+06"])
    x, info, _ = run(A, B, y)
    xo, io = oracle.alg1_solve(A, B, y)
    xc, _ = oracle.cr_solve(A, B, y)
    assert info["status"] == 0 == io["status"]
    assert rel_err(x, xo) <= 1e-10 and rel_err(x, xc) <= 1e-10


def test_refactor_and_resolve_reuse_the_plan(cuda_ok):
    N, m, k = 512, 8, 3
    plan = crs.Plan(N, m, k, flags=ALG1)
    for seed in (1, 2):
        A, B, y = synthetic.gen_system(N, m, k, seed=seed)
        dA, dB, dy = to_dev(A, B, y)
        crs.crsolve_factor(plan, dA, dB)
        for rhs in (y, 2 * y[:, :, ::-1].copy()):
            (dy,) = to_dev(rhs)
            x = crs.crsolve_solve(plan, dy).cpu().numpy()
            xo, _ = oracle.alg1_solve(A, B, rhs)
            assert rel_err(x, xo) <= TOL


def test_solve_host_buffers(cuda_ok):
    N, m, k = 256, 8, 4
    A, B, y = synthetic.gen_system(N, m, k, seed=17)
    plan = crs.Plan(N, m, k, flags=ALG1 | nat.CRSOLVE_PLAN_HOST_STAGING)
    tA, tB, ty = (torch.from_numpy(a).pin_memory() for a in (A, B, y))
    x, status = crs.crsolve_solve_host(plan, tA, tB, ty)
    xo, _ = oracle.alg1_solve(A, B, y)
    assert status == 0 and rel_err(x.numpy(), xo) <= TOL


def test_backward_matches_oracle(cuda_ok):
    N, m, k = 64, 4, 3
    A, B, y = synthetic.gen_system(N, m, k, seed=23)
    c = synthetic.gen_cotangent(N, m, k, seed=23)
    dA, dB, dy, dc = to_dev(A, B, y, c)
    dA.requires_grad_(True)
    dB.requires_grad_(True)
    dy.requires_grad_(True)
    x = crs.CRSolveFn.apply(dA, dB, dy, True, "alg1")
    loss = torch.real(torch.sum(torch.conj(dc) * x))
    loss.backward()
    xo, _ = oracle.alg1_solve(A, B, y)
    gy, gA, gB, st = oracle.cr_backward(A, B, xo, c)
    assert st == 0
    assert rel_err(dy.grad, gy) <= TOL
    assert rel_err(dA.grad, gA) <= TOL
    assert rel_err(dB.grad, gB) <= TOL


def test_method_argument(cuda_ok):
    A, B, y = synthetic.gen_system(32, 4, 2, seed=2)
    dA, dB, dy = to_dev(A, B, y)
    x = crs.solve(dA, dB, dy, method="alg1").cpu().numpy()
    xo, _ = oracle.alg1_solve(A, B, y)
    assert rel_err(x, xo) <= TOL
    with pytest.raises(ValueError):
        crs.solve(dA, dB, dy, method="pcr")
    A6, B6, y6 = synthetic.gen_system(6, 4, 2, seed=2)
    dA6, dB6, dy6 = to_dev(A6, B6, y6)
    with pytest.raises(RuntimeError):
        crs.solve(dA6, dB6, dy6, method="alg1")


# ------------------------------------------------------------------ full size
# N = 2^20, m = 8, k = 4 in the launch configuration bench.py times.

@pytest.mark.slow
def test_full_size_matches_oracles(cuda_ok):
    A, B, y = synthetic.gen_system(1 << 20, 8, 4, seed=1000)
    x, info, _ = run(A, B, y)
    assert info["status"] == 0
    xc, _ = oracle.cr_solve(A, B, y)
    assert rel_err(x, xc) <= TOL
    xo, io = oracle.alg1_solve(A, B, y)      # about half a minute on the host cores
    assert io["status"] == 0
    assert rel_err(x, xo) <= TOL


@pytest.mark.slow
def test_full_size_indefinite_flag(cuda_ok):
    """A_{N/2} - 3I at N = 2^20: Algorithm 1 factors A_{N/2} itself at depth 0."""
    A, B, y = synthetic.gen_system(1 << 20, 8, 4, seed=1000)
    A = synthetic.make_indefinite(A)
    assert np.linalg.eigvalsh(herm_from_lower(A[(1 << 19) - 1])).min() < 0
    x, info, _ = run(A, B, y)
    assert info == {"status": 1, "level": 0, "block": 1 << 19, "orig_block": 1 << 19}
    assert np.isnan(x).all()
