"""Pins for the oracle of the paper's Algorithm 1 (Sec. 3), which splits every
system into its odd half (U, E, u) and its even half (V, F, v) of eq. Formulas
and recurses on both.

Each test fixes ``oracle.alg1_solve`` / ``oracle.alg1_split`` to something
other than themselves: a hand-worked split, the dense Schur complements onto
the odd and the even unknowns, the dense LAPACK solve, closed forms, the
positive-definiteness test by eigenvalues, and the breakdown location found
by brute force from dense Schur complements (the quotient property: the
subsystem at depth d that holds the unknowns i = s (mod 2^d) is the Schur
complement of the whole matrix onto them).
"""
import os

import numpy as np
import pytest

import oracle
import synthetic
from tests.oracle_helpers import (assemble, brute_force_first_failure, dense_schur, dense_solve, eta_inf,
                                  herm_from_lower, rel_err)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, re, im = line.split()
                vals[key] = complex(float(re), float(im))
    return vals


def test_hand_worked_split_n2_m1():
    """N = 2, m = 1 by hand (tests/golden/alg1_n2_m1_by_hand.txt)."""
    g = _read_golden("alg1_n2_m1_by_hand.txt")
    A = np.array([[[g["A1"]]], [[g["A2"]]]])
    B = np.array([[[g["B1"]]]])
    y = np.array([[[g["y1"]]], [[g["y2"]]]])
    s = oracle.alg1_split(A, B, y)
    assert s["fail"] == 0
    for key in ("U", "u", "V", "v"):
        assert abs(s[key][0, 0, 0] - g[key + "1"]) <= 1e-15, key
    x, info = oracle.alg1_solve(A, B, y)
    assert info["status"] == 0
    assert abs(x[0, 0, 0] - g["x1"]) <= 1e-15 and abs(x[1, 0, 0] - g["x2"]) <= 1e-15


@pytest.mark.parametrize("N", [2, 4, 8, 16])
@pytest.mark.parametrize("m,k", [(1, 1), (3, 2), (5, 3)])
def test_split_equals_dense_schur_complements(N, m, k):
    """eq. Formulas: the odd system is the Schur complement onto the odd
    unknowns (even ones eliminated) and the even system the one onto the even
    unknowns; U/V on the block diagonal, E/F on the block sub-diagonal, u/v
    the eliminated right-hand sides."""
    A, B, y = synthetic.gen_system(N, m, k, seed=31 * N + m)
    D = assemble(A, B)
    Y = y.reshape(N * m, k)
    s = oracle.alg1_split(A, B, y)
    assert s["fail"] == 0
    h = N // 2
    for half, (Dg, Sb, rhs) in {0: ("U", "E", "u"), 1: ("V", "F", "v")}.items():
        keep = np.arange(half, N, 2)
        S, rows, rest = dense_schur(D, keep, m)
        Yr = Y[rows] - (D[np.ix_(rows, rest)] @ np.linalg.solve(D[np.ix_(rest, rest)], Y[rest]))
        scale = np.abs(S).max()
        for j in range(h):
            assert np.abs(s[Dg][j] - S[j * m:(j + 1) * m, j * m:(j + 1) * m]).max() <= 1e-14 * scale
            assert np.abs(s[rhs][j] - Yr[j * m:(j + 1) * m]).max() <= 1e-14 * np.abs(Yr).max()
            if j + 1 < h:
                assert np.abs(s[Sb][j] - S[(j + 1) * m:(j + 2) * m, j * m:(j + 1) * m]).max() <= 1e-14 * scale
                # nothing beyond the first block sub-diagonal
                if j + 2 < h:
                    assert np.abs(S[(j + 2) * m:(j + 3) * m, j * m:(j + 1) * m]).max() <= 1e-14 * scale


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("m,k", [(1, 1), (2, 3), (4, 1), (8, 2)])
def test_matches_dense_cholesky_solve(N, m, k):
    A, B, y = synthetic.gen_system(N, m, k, seed=7 * N + m)
    x, info = oracle.alg1_solve(A, B, y)
    assert info["status"] == 0
    assert rel_err(x, dense_solve(A, B, y)) <= 1e-13
    assert eta_inf(A, B, x, y) <= 1e-13


@pytest.mark.parametrize("N", [128, 1024])
def test_agrees_with_classic_reduction(N):
    """Both methods reach the exact x = A^{-1} y; they differ by rounding."""
    A, B, y = synthetic.gen_system(N, 4, 3, seed=N)
    x, info = oracle.alg1_solve(A, B, y)
    xc, infoc = oracle.cr_solve(A, B, y)
    assert info["status"] == 0 and infoc["status"] == 0
    assert rel_err(x, xc) <= 1e-13


@pytest.mark.parametrize("N", [1, 2, 8, 64])
def test_laplacian_closed_form(N):
    """1-D Laplacian (m = 1, A_j = 2, B_j = -1), y = e_1: x_i = (N+1-i)/(N+1)."""
    A = np.full((N, 1, 1), 2.0 + 0j)
    B = np.full((N - 1, 1, 1), -1.0 + 0j)
    y = np.zeros((N, 1, 1), np.complex128)
    y[0] = 1
    x, info = oracle.alg1_solve(A, B, y)
    i = np.arange(1, N + 1)
    assert info["status"] == 0
    # kappa ~ (2N/pi)^2; the error bound grows with it
    assert np.abs(x[:, 0, 0] - (N + 1 - i) / (N + 1)).max() <= 1e-15 * (N + 1) ** 2


def test_zero_coupling_is_blockwise_cholesky():
    A, B, y = synthetic.gen_system(16, 4, 2, seed=9)
    B = np.zeros_like(B)
    x, _ = oracle.alg1_solve(A, B, y)
    ref = np.stack([np.linalg.solve(herm_from_lower(A[j]), y[j]) for j in range(16)])
    assert rel_err(x, ref) <= 1e-14


def test_only_lower_triangle_and_real_diagonal_are_read():
    A, B, y = synthetic.gen_system(8, 4, 2, seed=5)
    x, _ = oracle.alg1_solve(A, B, y)
    A2 = A.copy()
    iu = np.triu_indices(4, 1)
    A2[:, iu[0], iu[1]] = 1e3 * (1 + 2j)
    A2[:, np.arange(4), np.arange(4)] += 7j
    x2, _ = oracle.alg1_solve(A2, B, y)
    assert np.array_equal(x, x2)


def test_rejects_n_not_power_of_two():
    A, B, y = synthetic.gen_system(6, 2, 1, seed=1)
    with pytest.raises(ValueError):
        oracle.alg1_solve(A, B, y)


def test_split_systems_are_bitwise_hermitian_and_positive_definite():
    """Sec. 4: with Cholesky-based products both halves are bit-wise Hermitian
    (and, as Schur complements of an HPD matrix, positive definite), at every
    depth of the recursion."""
    A, B, y = synthetic.gen_system(32, 5, 1, seed=11)
    todo = [(A, B)]
    depth = 0
    while todo and todo[0][0].shape[0] > 1:
        nxt = []
        for (Ad, Bd) in todo:
            s = oracle.alg1_split(Ad, Bd)
            assert s["fail"] == 0
            for Dg, Sb in (("U", "E"), ("V", "F")):
                for blk in s[Dg]:
                    assert np.array_equal(blk, blk.conj().T)
                    assert np.linalg.eigvalsh(blk).min() > 0
                nxt.append((s[Dg], s[Sb]))
        todo = nxt
        depth += 1
    assert depth == 5 and len(todo) == 32


def test_breakdown_iff_not_positive_definite_and_its_location():
    """Sec. 2 "Determination of Positive Definiteness": the recursion breaks
    down exactly when the matrix is not positive definite, and it does so at
    the first depth whose split systems hold a block that is not positive
    definite (found here by dense Schur complements)."""
    rng = np.random.default_rng(321)
    seen = {True: 0, False: 0}
    depths = set()
    for trial in range(150):
        N = 1 << int(rng.integers(0, 5))
        m = int(rng.integers(1, 4))
        A, B, y = synthetic.gen_system(N, m, 1, seed=2000 + trial, shift=0.2)
        lam = np.linalg.eigvalsh(assemble(A, B))
        tau = float(rng.uniform(0, 1.2 * lam.max()))
        A = A.copy()
        if rng.random() < 0.4:
            A = A - tau * np.eye(m)
        else:
            for b in rng.choice(N, size=int(rng.integers(1, N + 1)), replace=False):
                A[b] -= float(rng.uniform(0, tau)) * np.eye(m)
        lmin = np.linalg.eigvalsh(assemble(A, B)).min()
        if abs(lmin) < 1e-6 * lam.max():
            continue
        try:
            expect = brute_force_first_failure(A, B, 1e-9 * lam.max())
        except ValueError:
            continue
        _, info = oracle.alg1_solve(A, B, y)
        assert (info["status"] == 1) == (lmin < 0), (N, m, lmin, info)
        assert (expect is not None) == (lmin < 0)
        if expect is not None:
            assert (info["level"], info["orig_block"]) == expect, (N, m, info, expect)
            depths.add(expect[0])
        seen[lmin < 0] += 1
    assert seen[True] >= 10 and seen[False] >= 10
    assert len(depths) >= 3


def test_indefinite_diagonal_block_fails_at_depth_zero():
    """Algorithm 1 factors every A_i of the input system at depth 0, so an
    indefinite A_{N/2} is found there (classic reduction meets it only at its
    last level)."""
    N, m = 64, 8
    for seed in range(20):
        A, B, y = synthetic.gen_system(N, m, 1, seed=seed)
        Ai = synthetic.make_indefinite(A)
        if np.linalg.eigvalsh(herm_from_lower(Ai[N // 2 - 1])).min() < 0:
            break
    x, info = oracle.alg1_solve(Ai, B, y)
    assert info["status"] == 1 and info["level"] == 0 and info["orig_block"] == N // 2
    assert np.isnan(x).all()


def test_nan_input_reports_breakdown():
    A, B, y = synthetic.gen_system(8, 3, 1, seed=4)
    A[2, 1, 1] = np.nan
    x, info = oracle.alg1_solve(A, B, y)
    assert info["status"] == 1 and info["level"] == 0 and info["orig_block"] == 3
    assert np.isnan(x).all()
