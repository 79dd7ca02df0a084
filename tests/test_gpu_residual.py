"""GPU parity of the FP64 residual r = y - A x (crsolve_residual), the
residual of the mixed-precision form's iterative refinement.

Reference: the compensated residual of tests/oracle_helpers (pinned on the
CPU against rational arithmetic), i.e. the exact residual rounded.

Bound: the tensor-core method ("split": exact slice products; matrix entries
on a 60-bit per-row grid, x on a 54-bit per-column grid, pairs of slices
with i + j <= 11 kept, y - A x formed exactly and rounded once) has the
stated error bound per entry 2^-50 * K * max|row| * max|column| (K = 6m
real terms) plus the final rounding, the size of an FP64 dot product's
rounding error bound.
The FP64 method is held to the classical bound gamma_K * sum |a| |x|.
On integer data both must be exact.
"""
import numpy as np
import pytest
import torch

import synthetic
import paper_1807_00370_gb300 as crs
from tests.gpu_helpers import to_dev
from tests.oracle_helpers import coupling_blocks, residual_dd

pytestmark = pytest.mark.gpu


def _gpu(A, B, x, y, method):
    N = y.shape[0]
    dA, dB, dx, dy = to_dev(A, B if N > 1 else None, x, y)
    return crs.crsolve_residual(dA, dB, dx, dy, method=method).cpu().numpy()


def _bounds(A, B, x, y, rows):
    """Per entry (row i of block row j, column c): 2^-50 K max|row| max|col|
    plus two roundings for the split method, and (K + 1) u (|y| + sum |a||x|)
    over the K = 6m real terms for FP64."""
    N, m, k = x.shape
    split, fp64 = [], []
    for j in rows:
        blocks = coupling_blocks(A, B, j)
        Mr = np.concatenate(blocks, axis=1)                           # m x 3m complex
        X = np.concatenate([x[jb] if 0 <= jb < N else np.zeros((m, k), complex) for jb in (j - 1, j, j + 1)])
        rmax = np.maximum(np.abs(Mr.real), np.abs(Mr.imag)).max(axis=1)          # per row
        cmax = np.maximum(np.abs(X.real), np.abs(X.imag)).max(axis=0)            # per column
        K = 6 * m
        absum = (np.abs(Mr.real) + np.abs(Mr.imag)) @ (np.abs(X.real) + np.abs(X.imag))
        ay = np.maximum(np.abs(y[j].real), np.abs(y[j].imag))
        split.append(2.0 ** -50 * K * rmax[:, None] * cmax[None, :] + 2.0 ** -51 * (ay + absum) + 1e-300)
        fp64.append((K + 1) * 2.0 ** -53 * (ay + absum) * 1.01 + 1e-300)
    return np.array(split), np.array(fp64)


def _check(A, B, x, y, rows=None):
    N = y.shape[0]
    rows = list(range(N)) if rows is None else rows
    ref = residual_dd(A, B, x, y, rows)
    bs, bf = _bounds(A, B, x, y, rows)
    for method, bound in (("split", bs), ("split_image", bs), ("fp64", bf)):
        r = _gpu(A, B, x, y, method)[rows]
        for part in (np.real, np.imag):
            err = np.abs(part(r) - part(ref))
            assert np.all(err <= bound), (method, float((err / bound).max()))
    return ref


@pytest.mark.parametrize("N,m,k", [(1, 64, 32), (2, 64, 32), (5, 64, 32), (7, 40, 7), (3, 33, 33), (4, 8, 1),
                                   (6, 17, 65)])
def test_integer_data_is_exact(cuda_ok, N, m, k):
    """Integer entries with |v| < 2^10: every product and sum is exact in FP64,
    so both methods must return the exact residual bit for bit."""
    rng = np.random.default_rng(N * m + k)

    def ci(shape):
        return (rng.integers(-1000, 1000, shape) + 1j * rng.integers(-1000, 1000, shape)).astype(np.complex128)
    A, B, x, y = ci((N, m, m)), ci((max(N - 1, 0), m, m)), ci((N, m, k)), ci((N, m, k))
    ref = residual_dd(A, B, x, y)
    for method in ("split", "fp64"):
        assert np.array_equal(_gpu(A, B, x, y, method), ref), method


@pytest.mark.parametrize("N,m,k", [(3, 64, 32), (9, 64, 5), (5, 48, 40), (4, 33, 1), (6, 20, 9)])
def test_random_systems_within_the_fp64_bound(cuda_ok, N, m, k):
    A, B, y = synthetic.gen_system(N, m, k, seed=N + m + k)
    x = synthetic.gen_system(N, m, k, seed=N + m + k + 1)[2]
    _check(A, B, x, y)


def test_near_solution_cancellation(cuda_ok):
    """x close to A^{-1} y (the refinement's case): r is ~1e-7 of y, and the
    split residual still meets its bound against the exact residual."""
    import oracle
    A, B, y = synthetic.gen_system(8, 64, 32, seed=3)
    x, _ = oracle.cr_solve(A, B, y)
    x = x * (1 + 1e-7)
    _check(A, B, x, y)


def test_persistent_rows_and_wide_dynamic_range(cuda_ok):
    """More block rows than SMs (each CTA loops over several rows), rows and
    columns scaled by powers of two over a wide range; sampled rows against
    the compensated residual."""
    N, m, k = 400, 64, 32
    A, B, y = synthetic.gen_system(N, m, k, seed=11)
    x = synthetic.gen_system(N, m, k, seed=12)[2]
    rng = np.random.default_rng(1)
    sc = 2.0 ** rng.integers(-30, 30, N)
    A = A * sc[:, None, None]
    B = B * sc[1:, None, None]
    x = x * (2.0 ** rng.integers(-20, 20, k))[None, None, :]
    rows = [0, 1, 150, 151, 152, 153, 303, 398, 399]
    _check(A, B, x, y, rows)


def test_zero_and_non_finite_inputs(cuda_ok):
    """x = 0 gives r = y exactly; a NaN in column c of x_j makes column c of
    block rows j-1, j, j+1 NaN and leaves the rest finite."""
    N, m, k = 6, 64, 4
    A, B, y = synthetic.gen_system(N, m, k, seed=5)
    r0 = _gpu(A, B, np.zeros_like(y), y, "split")
    assert np.array_equal(r0, y)
    x = synthetic.gen_system(N, m, k, seed=6)[2]
    x[3, 10, 2] = np.nan
    r = _gpu(A, B, x, y, "split")
    bad = np.isnan(r.real) | np.isnan(r.imag)
    assert bad[2:5, :, 2].all()
    bad[2:5, :, 2] = False
    assert not bad.any()


@pytest.mark.parametrize("N,m,k", [(5, 64, 32), (160, 64, 33), (7, 40, 5), (1, 64, 32), (2, 33, 65), (305, 64, 32)])
def test_precomputed_matrix_slices_give_the_same_bits(cuda_ok, N, m, k):
    """"split_image" (matrix slices written once to the workspace and copied
    in by bulk copies, as the mixed form does) equals "split" bit for bit."""
    A, B, y = synthetic.gen_system(N, m, k, seed=N * k)
    x = synthetic.gen_system(N, m, k, seed=N * k + 1)[2]
    assert np.array_equal(_gpu(A, B, x, y, "split_image"), _gpu(A, B, x, y, "split"))
