"""GPU parity of the adjoint: crsolve_backward and CRSolveFn against the
oracle's adjoint, dense torch autograd, and central finite differences.

Tolerances: the re-solve has the forward solve's accuracy (1e-12 relative on
these kappa ~ 10 systems); the outer products add O(k) rounding.  Central
differences with h = 1e-6 carry O(h^2) truncation plus O(u/h) rounding, so
they are compared at 1e-6 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_1807_00370_gb300 as crs
from tests.gpu_helpers import rel_err, to_dev

pytestmark = pytest.mark.gpu


def _backward(A, B, y, c):
    N, m, k = y.shape
    dA, dB, dy, dc = to_dev(A, B if N > 1 else None, y, c)
    plan = crs.Plan(N, m, k)
    crs.crsolve_factor(plan, dA, dB)
    x = crs.crsolve_solve(plan, dy)
    gy, gA, gB = crs.crsolve_backward(plan, x, dc)
    return x, gy, gA, gB


@pytest.mark.parametrize("N,m,k", [(1, 3, 2), (2, 1, 1), (64, 4, 3), (1000, 16, 8), (77, 32, 5)])
def test_backward_matches_oracle_adjoint(cuda_ok, N, m, k):
    A, B, y = synthetic.gen_system(N, m, k, seed=N + m)
    c = synthetic.gen_cotangent(N, m, k, seed=N + m)
    x, gy, gA, gB = _backward(A, B, y, c)
    xo, _ = oracle.cr_solve(A, B, y)
    gyo, gAo, gBo, st = oracle.cr_backward(A, B, xo, c)
    assert st == 0
    assert rel_err(gy, gyo) <= 1e-12
    assert rel_err(gA, gAo) <= 1e-12
    gAh = gA.cpu().numpy()
    assert np.array_equal(gAh, np.conj(np.swapaxes(gAh, 1, 2)))   # exactly Hermitian
    if N > 1:
        assert rel_err(gB, gBo) <= 1e-12


def test_autograd_function_matches_dense_autograd(cuda_ok):
    N, m, k = 16, 4, 3
    A, B, y = synthetic.gen_system(N, m, k, seed=31)
    c = torch.from_numpy(synthetic.gen_cotangent(N, m, k, seed=31)).cuda()
    tA, tB, ty = (torch.from_numpy(a).cuda().requires_grad_() for a in (A, B, y))
    x = crs.CRSolveFn.apply(tA, tB, ty)
    torch.real(torch.sum(torch.conj(c) * x)).backward()
    rA, rB, ry = (torch.from_numpy(a).cuda().requires_grad_() for a in (A, B, y))
    D = torch.zeros((N * m, N * m), dtype=torch.complex128, device="cuda")
    for j in range(N):
        D[j * m:(j + 1) * m, j * m:(j + 1) * m] = 0.5 * (rA[j] + rA[j].conj().T)
        if j + 1 < N:
            D[(j + 1) * m:(j + 2) * m, j * m:(j + 1) * m] = rB[j]
            D[j * m:(j + 1) * m, (j + 1) * m:(j + 2) * m] = rB[j].conj().T
    xr = torch.linalg.solve(D, ry.reshape(N * m, k)).reshape(N, m, k)
    torch.real(torch.sum(torch.conj(c) * xr)).backward()
    assert rel_err(x.detach(), xr.detach().cpu().numpy()) <= 1e-12
    for g, r in ((tA.grad, rA.grad), (tB.grad, rB.grad), (ty.grad, ry.grad)):
        assert rel_err(g, r.cpu().numpy()) <= 1e-12


@pytest.mark.slow
def test_full_size_adjoint_against_oracle_and_central_differences(cuda_ok):
    """N = 2^16, m = 16, k = 8; loss = Re sum(conj(c) * x)."""
    N, m, k = 1 << 16, 16, 8
    A, B, y = synthetic.gen_system(N, m, k, seed=2000)
    c = synthetic.gen_cotangent(N, m, k, seed=2000)
    x, gy, gA, gB = _backward(A, B, y, c)
    xo, _ = oracle.cr_solve(A, B, y)
    gyo, gAo, gBo, _ = oracle.cr_backward(A, B, xo, c)
    assert rel_err(x, xo) <= 1e-12
    assert rel_err(gy, gyo) <= 1e-12 and rel_err(gA, gAo) <= 1e-12 and rel_err(gB, gBo) <= 1e-12
    dA, dB, dy, dc = to_dev(A, B, y, c)
    plan = crs.Plan(N, m, k)

    def loss(a, b, yy):
        crs.crsolve_factor(plan, a, b)
        return float(torch.real(torch.sum(torch.conj(dc) * crs.crsolve_solve(plan, yy))).item())

    gen = torch.Generator(device="cuda").manual_seed(7)

    def cn(shape):
        return torch.view_as_complex(torch.randn(tuple(shape) + (2,), generator=gen, device="cuda",
                                                 dtype=torch.float64) * np.sqrt(0.5))

    h = 1e-6
    for _ in range(4):
        pA = cn(dA.shape)
        pA = 0.5 * (pA + pA.conj().transpose(1, 2))
        pB, py = cn(dB.shape), cn(dy.shape)
        fd = (loss(dA + h * pA, dB + h * pB, dy + h * py) - loss(dA - h * pA, dB - h * pB, dy - h * py)) / (2 * h)
        an = float(torch.real(torch.sum(torch.conj(gA) * pA) + torch.sum(torch.conj(gB) * pB)
                              + torch.sum(torch.conj(gy) * py)).item())
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_gradients_are_nan_after_breakdown(cuda_ok):
    A, B, y = synthetic.gen_system(32, 4, 2, seed=5)
    A[7] -= 60.0 * np.eye(4)
    c = synthetic.gen_cotangent(32, 4, 2, seed=5)
    x, gy, gA, gB = _backward(A, B, y, c)
    assert torch.isnan(gy).all() and torch.isnan(gA).all() and torch.isnan(gB).all()


def test_recomputed_factors_give_identical_gradients(cuda_ok):
    """keep_factors=False frees the plan after the forward pass and re-factors
    in the backward pass; the gradients are bit-identical."""
    N, m, k = 200, 8, 3
    A, B, y = synthetic.gen_system(N, m, k, seed=77)
    c = torch.from_numpy(synthetic.gen_cotangent(N, m, k, seed=77)).cuda()
    grads = []
    for keep in (True, False):
        tA, tB, ty = (torch.from_numpy(a).cuda().requires_grad_() for a in (A, B, y))
        x = crs.CRSolveFn.apply(tA, tB, ty, keep)
        torch.real(torch.sum(torch.conj(c) * x)).backward()
        grads.append((tA.grad, tB.grad, ty.grad))
    for g1, g2 in zip(*grads):
        assert torch.equal(g1, g2)
