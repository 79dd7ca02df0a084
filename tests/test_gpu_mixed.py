"""GPU parity of the mixed-precision form (FP32 fine levels, FP64 coarse
levels, FP64 residual and iterative refinement) against the FP64 oracle.

Bound: relative error <= 1e-10 against the oracle (the stated target), on
systems with kappa up to ~1e6 (shifts from tests/golden/kappa_shifts.json).
Breakdown flags must equal the oracle's (the mixed form re-decides any FP32
breakdown in FP64).
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

pytestmark = pytest.mark.gpu
BOUND = 1e-10
SHIFTS = os.path.join(os.path.dirname(__file__), "golden", "kappa_shifts.json")


def _mixed(A, B, y, flags=0):
    N, m, k = y.shape
    dA, dB, dy = to_dev(A, B if N > 1 else None, y)
    plan = crs.Plan(N, m, k, precision=nat.CRSOLVE_MIXED, flags=flags)
    crs.crsolve_factor(plan, dA, dB)
    x = crs.crsolve_solve(plan, dy)
    return x.cpu().numpy(), crs.crsolve_info_get(plan), crs.crsolve_mixed_stats(plan)


@pytest.mark.parametrize("N,m,k", [(1, 4, 1), (2, 3, 2), (65, 4, 1), (300, 8, 4), (1000, 16, 8), (257, 64, 32),
                                   (4097, 5, 3), (129, 32, 16), (77, 40, 3), (200, 57, 20)])
def test_mixed_matches_oracle(cuda_ok, N, m, k):
    A, B, y = synthetic.gen_system(N, m, k, seed=N * m + k)
    x, info, st = _mixed(A, B, y)
    xo, io = oracle.cr_solve(A, B, y)
    assert info == io and info["status"] == 0
    err = rel_err(x, xo)
    assert err <= BOUND, (err, st)
    if N > 64:
        assert not st["fp64_fallback"] and st["iterations"] <= 4, st


@pytest.mark.parametrize("N,m", [(512, 8), (96, 40), (64, 64)])
def test_mixed_breakdown_flags_equal_fp64(cuda_ok, N, m):
    for seed in range(20):
        A, B, y = synthetic.gen_system(N, m, 2, seed=seed)
        Ai = synthetic.make_indefinite(A)
        if np.linalg.eigvalsh(Ai[N // 2 - 1]).min() < 0:
            break
    x, info, st = _mixed(Ai, B, y)
    _, io = oracle.cr_solve(Ai, B, y)
    assert info == io and info["status"] == 1
    assert np.isnan(x).all()


def _kappa_case(name, kappa):
    if not os.path.exists(SHIFTS):
        pytest.skip("kappa_shifts.json missing (run tests/golden/make_kappa_shifts.py)")
    case = json.load(open(SHIFTS)).get(name)
    if case is None:
        pytest.skip(f"{name} not in kappa_shifts.json")
    return case, case["shifts"][f"{kappa:.0e}"]


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
def test_mixed_at_controlled_kappa(cuda_ok, kappa):
    """N = 2^10, m = 64, k = 32 with the diagonal shift that gives kappa."""
    case, shift = _kappa_case("mixed_N2p10_m64_k32", kappa)
    A, B, y = synthetic.gen_system(case["N"], case["m"], case["k"], case["seed"], shift=shift)
    x, info, st = _mixed(A, B, y)
    xo, io = oracle.cr_solve(A, B, y)
    assert info == io and info["status"] == 0
    err = rel_err(x, xo)
    print(f"kappa~{kappa:.0e}: rel err vs oracle {err:.2e}, stats {st}")
    assert err <= BOUND, (err, st)
    # the conjugate-gradient refinement converges in mixed precision at every kappa
    assert not st["fp64_fallback"], st


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_mixed_with_fp64_pipe_residuals(cuda_ok, kappa):
    """The same refinement with every residual and product on the FP64 pipe
    (CRSOLVE_PLAN_FP64_RESIDUAL) instead of the tensor-core splitting."""
    case, shift = _kappa_case("mixed_N2p10_m64_k32", kappa)
    A, B, y = synthetic.gen_system(case["N"], case["m"], case["k"], case["seed"], shift=shift)
    x, info, st = _mixed(A, B, y, flags=nat.CRSOLVE_PLAN_FP64_RESIDUAL)
    xo, io = oracle.cr_solve(A, B, y)
    assert info == io and info["status"] == 0
    assert rel_err(x, xo) <= BOUND, st
    assert not st["fp64_fallback"], st


def test_plain_fp64_at_kappa_1e6(cuda_ok):
    """The FP64 path on the kappa ~ 1e6 variant of the m = 8, k = 4 workload (N = 2^12)."""
    case, shift = _kappa_case("plain_N2p12_m8_k4", 1e6)
    A, B, y = synthetic.gen_system(case["N"], case["m"], case["k"], case["seed"], shift=shift)
    dA, dB, dy = to_dev(A, B, y)
    plan = crs.Plan(case["N"], case["m"], case["k"])
    crs.crsolve_factor(plan, dA, dB)
    x = crs.crsolve_solve(plan, dy).cpu().numpy()
    xo, _ = oracle.cr_solve(A, B, y)
    assert rel_err(x, xo) <= BOUND


# The FP32 preconditioner alone (crsolve_mixed_precondition): one FP32 solve,
# no refinement.  For the class 33 <= m <= 64 its sweeps are the L^{-1}
# products of cr_solve32.cu: column chunks of 8 (k <= 8), 16 and 32, ragged
# last chunks (k = 20, 40), odd m (8-byte copies of L^{-1}) and odd k (8-byte
# copies of the right-hand sides), N from 3 (one FP32 level) up.  Bound: the
# FP32 solve's forward error, at most c kappa u_32 with u_32 = 2^-24; these
# synthetic systems have kappa < 1e2, so 1e-4 leaves c ~ 170.
PRECOND_BOUND = 1e-4


@pytest.mark.parametrize("N,m,k", [(3, 64, 32), (257, 64, 32), (77, 40, 3), (200, 57, 20), (129, 33, 1),
                                   (300, 64, 40), (64, 48, 9), (1000, 16, 8), (513, 61, 16)])
def test_mixed_preconditioner_matches_oracle(cuda_ok, N, m, k):
    A, B, y = synthetic.gen_system(N, m, k, seed=7 * N + m + k)
    dA, dB, dy = to_dev(A, B if N > 1 else None, y)
    plan = crs.Plan(N, m, k, precision=nat.CRSOLVE_MIXED)
    crs.crsolve_factor(plan, dA, dB)
    z = crs.crsolve_mixed_precondition(plan, dy)
    xo, io = oracle.cr_solve(A, B, y)
    assert io["status"] == 0
    err = rel_err(z.cpu().numpy(), xo)
    assert err <= PRECOND_BOUND, err
    # in place (r and z the same buffer) gives the same bits
    dz = dy.clone()
    crs.crsolve_mixed_precondition(plan, dz, dz)
    assert torch.equal(dz, z)


def test_mixed_preconditioner_rejects_fp64_plans(cuda_ok):
    N, m, k = 64, 40, 4
    A, B, y = synthetic.gen_system(N, m, k, seed=5)
    dA, dB, dy = to_dev(A, B, y)
    plan = crs.Plan(N, m, k)
    crs.crsolve_factor(plan, dA, dB)
    with pytest.raises(RuntimeError, match="unsupported"):
        crs.crsolve_mixed_precondition(plan, dy)


def test_mixed_full_size_at_kappa_1e6(cuda_ok):
    """The precision workload at its full size (N = 2^14, m = 64, k = 32) and
    the hardest conditioning (κ ≈ 1e6), as the benchmark runs it: the refined
    solution against the oracle on the whole system, within the stated 1e-10,
    with no FP64 handover."""
    case, shift = _kappa_case("mixed_N2p14_m64_k32", 1e6)
    A, B, y = synthetic.gen_system(case["N"], case["m"], case["k"], case["seed"], shift=shift)
    x, info, st = _mixed(A, B, y)
    xo, io = oracle.cr_solve(A, B, y)
    assert info == io and info["status"] == 0
    err = rel_err(x, xo)
    print(f"N=2^14 m=64 k=32 kappa~1e6: rel err vs oracle {err:.2e}, stats {st}")
    assert err <= BOUND, (err, st)
    assert not st["fp64_fallback"], st
