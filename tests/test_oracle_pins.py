"""Pins for the CPU oracle against facts fixed by the mathematics and the paper.

Each test fixes the oracle to something other than itself: a dense LAPACK
solve, a closed form, a hand-worked example, a textbook special case, the
dense Schur complement, or an eigenvalue test of positive definiteness.
"""
import os

import numpy as np
import pytest

import oracle
import synthetic
from tests.oracle_helpers import (assemble, brute_force_first_failure_classic, dense_solve, eta_inf,
                                  herm_from_lower, rel_err, shift_blocks)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 8, 16, 33, 64])
@pytest.mark.parametrize("m,k", [(1, 1), (2, 3), (4, 1), (8, 2)])
def test_matches_dense_cholesky_solve(N, m, k):
    """Whole solve equals the dense LAPACK solve of the assembled eq. Axb."""
    A, B, y = synthetic.gen_system(N, m, k, seed=100 * N + m)
    x, info = oracle.cr_solve(A, B, y)
    assert info["status"] == 0
    ref = dense_solve(A, B, y)
    assert rel_err(x, ref) <= 1e-13
    assert eta_inf(A, B, x, y) <= 1e-13


def test_matvec_is_the_dense_product():
    A, B, y = synthetic.gen_system(19, 5, 3, seed=3)
    D = assemble(A, B)
    out = oracle.matvec(A, B, y)
    ref = (D @ y.reshape(-1, 3)).reshape(y.shape)
    assert np.abs(out - ref).max() <= 1e-14 * np.abs(ref).max()


def test_only_lower_triangle_and_real_diagonal_are_read():
    A, B, y = synthetic.gen_system(9, 4, 2, seed=5)
    x, _ = oracle.cr_solve(A, B, y)
    A2 = A.copy()
    iu = np.triu_indices(4, 1)
    A2[:, iu[0], iu[1]] = 1e3 * (1 + 2j)          # garbage in the strict upper triangle
    A2[:, np.arange(4), np.arange(4)] += 7j        # imaginary part on the diagonal
    x2, _ = oracle.cr_solve(A2, B, y)
    assert np.array_equal(x, x2)


def test_hand_worked_n2_m1():
    """N = 2, m = 1 by hand from eq. Formulas (tests/golden/n2_m1_by_hand.txt)."""
    vals = {}
    with open(os.path.join(GOLDEN, "n2_m1_by_hand.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, re, im = line.split()
                vals[name] = complex(float(re), float(im))
    A = np.array([[[vals["A1"]]], [[vals["A2"]]]])
    B = np.array([[[vals["B1"]]]])
    y = np.array([[[vals["y1"]]], [[vals["y2"]]]])
    lev = oracle.cr_level(A, B, y)
    assert abs(lev["An"][0, 0, 0] - vals["V1"]) <= 1e-15
    assert abs(lev["yn"][0, 0, 0] - vals["v1"]) <= 1e-15
    x, info = oracle.cr_solve(A, B, y)
    assert info["status"] == 0
    assert abs(x[0, 0, 0] - vals["x1"]) <= 1e-15
    assert abs(x[1, 0, 0] - vals["x2"]) <= 1e-15


@pytest.mark.parametrize("N", [1, 2, 3, 10, 31, 64, 257])
def test_laplacian_closed_form(N):
    """m = 1, A_j = 2, B_j = -1, y = e_1: x_i = (N + 1 - i) / (N + 1)."""
    A = np.full((N, 1, 1), 2.0 + 0j)
    B = np.full((N - 1, 1, 1), -1.0 + 0j)
    y = np.zeros((N, 1, 1), np.complex128)
    y[0] = 1.0
    x, info = oracle.cr_solve(A, B, y)
    i = np.arange(1, N + 1)
    ref = (N + 1 - i) / (N + 1)
    assert info["status"] == 0
    # kappa ~ (2N/pi)^2; the error bound grows with it
    assert np.abs(x[:, 0, 0] - ref).max() <= 1e-15 * (N + 1) ** 2


@pytest.mark.parametrize("N,m,s", [(16, 3, 0.7), (37, 4, -0.45 + 0.2j)])
def test_kronecker_case_reduces_to_scalar_tridiagonal(N, m, s):
    """A_j = T, B_j = s I: in T's eigenbasis the system splits into m scalar
    tridiagonal systems (diagonal lambda_q, off-diagonals s and conj(s)),
    each solved here by scipy's banded Hermitian solver."""
    from scipy.linalg import solveh_banded
    rng = np.random.default_rng(7)
    G = synthetic.cn(rng, (m, m))
    T = G @ G.conj().T / m + 3.0 * np.eye(m)
    lam, U = np.linalg.eigh(T)
    A = np.broadcast_to(T, (N, m, m)).copy()
    B = np.broadcast_to(s * np.eye(m), (N - 1, m, m)).copy()
    y = synthetic.cn(rng, (N, m, 2))
    x, info = oracle.cr_solve(A, B, y)
    assert info["status"] == 0
    yt = np.einsum("qa,jak->jqk", U.conj().T, y)       # U^H y_j
    xt = np.empty_like(yt)
    for q in range(m):
        ab = np.zeros((2, N), np.complex128)            # upper form: ab[0,1:] = superdiagonal
        ab[0, 1:] = np.conj(s)                          # (j, j+1) entry is B_j^H = conj(s)
        ab[1, :] = lam[q]
        xt[:, q, :] = solveh_banded(ab, yt[:, q, :])
    ref = np.einsum("aq,jqk->jak", U, xt)
    assert rel_err(x, ref) <= 1e-13


def test_zero_coupling_is_blockwise_cholesky():
    A, B, y = synthetic.gen_system(13, 6, 2, seed=11)
    B = np.zeros_like(B)
    x, _ = oracle.cr_solve(A, B, y)
    ref = np.stack([np.linalg.solve(herm_from_lower(A[j]), y[j]) for j in range(13)])
    assert rel_err(x, ref) <= 1e-14


def test_single_block_is_cholesky_solve():
    A, B, y = synthetic.gen_system(1, 7, 3, seed=2)
    x, info = oracle.cr_solve(A, B, y)
    assert info["status"] == 0
    assert rel_err(x[0], np.linalg.solve(A[0], y[0])) <= 1e-14


def _paper_reordering(A, B, y):
    """D1, D2, C, y_o, y_e of the odd-then-even reordering (Sec. 2), dense."""
    N, m, k = y.shape
    D = assemble(A, B)
    odd = [j for j in range(N) if j % 2 == 0]      # 1-based 1, 3, 5, ...
    even = [j for j in range(N) if j % 2 == 1]     # 1-based 2, 4, 6, ...
    io = np.concatenate([np.arange(j * m, (j + 1) * m) for j in odd])
    ie = np.concatenate([np.arange(j * m, (j + 1) * m) for j in even])
    Y = y.reshape(N * m, k)
    return D[np.ix_(io, io)], D[np.ix_(ie, ie)], D[np.ix_(ie, io)], Y[io], Y[ie]


@pytest.mark.parametrize("N", [2, 3, 4, 9, 16])
def test_level_equals_dense_schur_complement(N):
    """V = D2 - C D1^{-1} C^H and v = y_e - C D1^{-1} y_o (eq. even) against
    the oracle's reduced system."""
    m, k = 3, 2
    A, B, y = synthetic.gen_system(N, m, k, seed=N)
    D1, D2, C, yo, ye = _paper_reordering(A, B, y)
    V = D2 - C @ np.linalg.solve(D1, C.conj().T)
    v = ye - C @ np.linalg.solve(D1, yo)
    lev = oracle.cr_level(A, B, y)
    ne = N // 2
    Vd = np.zeros_like(V)
    for j in range(ne):
        Vd[j * m:(j + 1) * m, j * m:(j + 1) * m] = lev["An"][j]
        if j + 1 < ne:
            Vd[(j + 1) * m:(j + 2) * m, j * m:(j + 1) * m] = lev["Bn"][j]
            Vd[j * m:(j + 1) * m, (j + 1) * m:(j + 2) * m] = lev["Bn"][j].conj().T
    assert np.abs(Vd - V).max() <= 1e-14 * np.abs(V).max()
    assert np.abs(lev["yn"].reshape(ne * m, k) - v).max() <= 1e-14 * np.abs(v).max()
    # the factor outputs themselves: L L^H = A_odd, L P = B_{i-1}, L Q = B_i^H
    for t in range((N + 1) // 2):
        c = 2 * t
        Lt = lev["L"][t]
        assert np.allclose(Lt @ Lt.conj().T, herm_from_lower(A[c]), rtol=0, atol=1e-14 * 10)
        if c >= 1:
            assert np.abs(Lt @ lev["P"][t] - B[c - 1]).max() <= 1e-14
        if c + 1 < N:
            assert np.abs(Lt @ lev["Q"][t] - B[c].conj().T).max() <= 1e-14


def test_reduced_blocks_are_bitwise_hermitian_and_positive_definite():
    """Sec. 4: with Cholesky products the reduced blocks are bit-wise Hermitian;
    Sec. 2: Schur complements of an HPD matrix are HPD."""
    A, B, y = synthetic.gen_system(45, 5, 2, seed=9)
    while A.shape[0] > 1:
        lev = oracle.cr_level(A, B, y)
        An, Bn = lev["An"], lev["Bn"]
        assert np.array_equal(An, np.conj(np.swapaxes(An, 1, 2)))
        assert np.linalg.eigvalsh(assemble(An, Bn)).min() > 0
        A, B, y = An, Bn, lev["yn"]


@pytest.mark.parametrize("N", [1, 2, 5, 6, 13, 33, 100])
def test_general_n_equals_padded_power_of_two(N):
    """Reading for N not a power of two: padding with decoupled identity
    blocks (A = I, B = 0, y = 0) to 2^ceil(log2 N) leaves x unchanged."""
    m, k = 3, 2
    A, B, y = synthetic.gen_system(N, m, k, seed=N + 1)
    x, _ = oracle.cr_solve(A, B, y)
    P = 1 << max(0, (N - 1).bit_length())
    Ap = np.broadcast_to(np.eye(m, dtype=np.complex128), (P, m, m)).copy()
    Ap[:N] = A
    Bp = np.zeros((P - 1, m, m), np.complex128)
    Bp[:N - 1] = B
    yp = np.zeros((P, m, k), np.complex128)
    yp[:N] = y
    xp, _ = oracle.cr_solve(Ap, Bp, yp)
    assert rel_err(x, xp[:N]) <= 1e-14
    assert np.abs(xp[N:]).max(initial=0.0) == 0.0


def test_breakdown_iff_not_positive_definite():
    """Sec. 2 and Sec. 4: the method breaks down exactly when the matrix is not
    positive definite.  Random tiny cases with an eigenvalue margin."""
    rng = np.random.default_rng(123)
    seen = {True: 0, False: 0}
    for trial in range(120):
        N = int(rng.integers(1, 17))
        m = int(rng.integers(1, 5))
        A, B, y = synthetic.gen_system(N, m, 1, seed=1000 + trial, shift=0.2)
        lam = np.linalg.eigvalsh(assemble(A, B))
        # shift the whole matrix, or only one diagonal block, by tau
        tau = float(rng.uniform(0, 1.5 * lam.max()))
        if rng.random() < 0.5:
            A = A - tau * np.eye(m)
        else:
            A = A.copy()
            A[int(rng.integers(0, N))] -= tau * np.eye(m)
        lmin = np.linalg.eigvalsh(assemble(A, B)).min()
        if abs(lmin) < 1e-6 * lam.max():
            continue
        _, info = oracle.cr_solve(A, B, y)
        assert (info["status"] == 1) == (lmin < 0), (N, m, lmin, info)
        seen[lmin < 0] += 1
    assert seen[True] >= 10 and seen[False] >= 10


@pytest.mark.parametrize("p,m", [(3, 2), (6, 8), (9, 4)])
def test_predicted_breakdown_location(p, m):
    """A_{N/2} - 3I with N = 2^p: block N/2 stays even until level p-1, where
    it is local block 1 of a 2-block system; every earlier pivot belongs to a
    Schur complement of an unmodified HPD principal submatrix.  So the first
    breakdown is (level p-1, block 1, original block N/2) provided
    A_{N/2} - 3I is itself indefinite."""
    N = 1 << p
    for seed in range(20):
        A, B, y = synthetic.gen_system(N, m, 1, seed=seed)
        Ai = synthetic.make_indefinite(A)
        if np.linalg.eigvalsh(herm_from_lower(Ai[N // 2 - 1])).min() < 0:
            break
    _, info = oracle.cr_solve(Ai, B, y)
    assert info == {"status": 1, "level": p - 1, "block": 1, "orig_block": N // 2}


@pytest.mark.parametrize("N,m,blocks,expect", [
    (16, 3, [11, 5, 3], (0, 3)),     # three odd blocks of level 0 fail: the smallest is reported
    (32, 2, [20, 12], (2, 3)),       # originals 4*5 and 4*3: even at levels 0 and 1, odd blocks 5, 3 of level 2
    (37, 4, [37, 9, 25], (0, 9)),    # odd N, the last block (left neighbour only) among the failures
    (24, 3, [24, 8], (3, 1)),        # level 3 has 3 blocks (originals 8, 16, 24): blocks 1 and 3 fail
    (32, 2, [12, 27], (0, 27)),      # the first level decides before the index: 27 fails at level 0, 12 at 2
])
def test_breakdown_tie_break_smallest_block_of_first_level(N, m, blocks, expect):
    """Sec. 2 "Determination of Positive Definiteness": a breakdown means the
    matrix is not positive definite.  Reading for the location when several
    odd blocks of one level fail: the first level with a failure, then the
    smallest 1-based local block there.  The expected location is set by
    construction (each shifted block is indefinite on its own, and its
    reduced block is that block minus positive semidefinite Schur terms) and
    confirmed by brute force on the dense matrix (every failing odd block of
    the first failing level, from Schur complements, no reduction step)."""
    A, B, y = synthetic.gen_system(N, m, 1, seed=N + 7 * m)
    A = shift_blocks(A, blocks)
    level, block, fails = brute_force_first_failure_classic(A, B, margin=1e-6)
    assert (level, block) == expect
    assert len(fails) >= 2 or N == 32 and blocks == [12, 27]
    x, info = oracle.cr_solve(A, B, y)
    assert info == {"status": 1, "level": level, "block": block, "orig_block": block << level}
    assert np.isnan(x).all()


def test_breakdown_tie_break_random_multi_failures():
    """Random tiny systems with several shifted diagonal blocks: the oracle's
    (level, block) equals the brute-force first failure, and at least a few
    dozen cases have two or more failing odd blocks at that level."""
    rng = np.random.default_rng(2024)
    multi = 0
    for trial in range(240):
        N = int(rng.integers(2, 33))
        m = int(rng.integers(1, 5))
        A, B, y = synthetic.gen_system(N, m, 1, seed=7000 + trial, shift=0.3)
        A = A.copy()
        for b in rng.choice(np.arange(N), size=min(int(rng.integers(2, 7)), N), replace=False):
            A[b] -= float(rng.uniform(0.5, 4.0)) * np.eye(m)
        try:
            bf = brute_force_first_failure_classic(A, B, margin=1e-6)
        except ValueError:
            continue
        _, info = oracle.cr_solve(A, B, y)
        if bf is None:
            assert info["status"] == 0, (trial, info)
            continue
        level, block, fails = bf
        assert info == {"status": 1, "level": level, "block": block, "orig_block": block << level}, (trial, bf)
        multi += len(fails) >= 2
    assert multi >= 30, multi


def test_nan_input_reports_breakdown():
    A, B, y = synthetic.gen_system(8, 3, 1, seed=4)
    A[2, 1, 1] = np.nan
    x, info = oracle.cr_solve(A, B, y)
    assert info["status"] == 1 and info["level"] == 0 and info["block"] == 3
    assert np.isnan(x).all()


# ---------------------------------------------------------------- adjoint

def _loss(A, B, y, c):
    x, _ = oracle.cr_solve(A, B, y)
    return float(np.real(np.sum(np.conj(c) * x)))


def test_backward_matches_central_differences():
    N, m, k = 12, 3, 2
    A, B, y = synthetic.gen_system(N, m, k, seed=21)
    c = synthetic.gen_cotangent(N, m, k, seed=21)
    x, _ = oracle.cr_solve(A, B, y)
    gy, gA, gB, st = oracle.cr_backward(A, B, x, c)
    assert st == 0
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(4):
        dA = synthetic.cn(rng, A.shape)
        dA = 0.5 * (dA + np.conj(np.swapaxes(dA, 1, 2)))          # Hermitian direction
        dB = synthetic.cn(rng, B.shape)
        dy = synthetic.cn(rng, y.shape)
        fd = (_loss(A + h * dA, B + h * dB, y + h * dy, c)
              - _loss(A - h * dA, B - h * dB, y - h * dy, c)) / (2 * h)
        an = float(np.real(np.sum(np.conj(gA) * dA) + np.sum(np.conj(gB) * dB)
                           + np.sum(np.conj(gy) * dy)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_backward_matches_dense_torch_autograd():
    torch = pytest.importorskip("torch")
    N, m, k = 16, 4, 3
    A, B, y = synthetic.gen_system(N, m, k, seed=31)
    c = synthetic.gen_cotangent(N, m, k, seed=31)
    x, _ = oracle.cr_solve(A, B, y)
    gy, gA, gB, _ = oracle.cr_backward(A, B, x, c)
    tA = torch.tensor(A, requires_grad=True)
    tB = torch.tensor(B, requires_grad=True)
    ty = torch.tensor(y, requires_grad=True)
    D = torch.zeros((N * m, N * m), dtype=torch.complex128)
    for j in range(N):
        D[j * m:(j + 1) * m, j * m:(j + 1) * m] = 0.5 * (tA[j] + tA[j].conj().T)
        if j + 1 < N:
            D[(j + 1) * m:(j + 2) * m, j * m:(j + 1) * m] = tB[j]
            D[j * m:(j + 1) * m, (j + 1) * m:(j + 2) * m] = tB[j].conj().T
    tx = torch.linalg.solve(D, ty.reshape(N * m, k))
    loss = torch.real(torch.sum(torch.conj(torch.tensor(c).reshape(N * m, k)) * tx))
    loss.backward()
    assert np.abs(tA.grad.numpy() - gA).max() <= 1e-12
    assert np.abs(tB.grad.numpy() - gB).max() <= 1e-12
    assert np.abs(ty.grad.numpy() - gy).max() <= 1e-12
