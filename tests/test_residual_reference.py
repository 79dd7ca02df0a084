"""CPU pins of the compensated residual that the GPU residual tests compare
against: exact on integer data, and equal to the correctly rounded exact
residual (rational arithmetic) on random data."""
from fractions import Fraction

import numpy as np

import oracle
import synthetic
from tests.oracle_helpers import coupling_blocks, residual_dd


def _exact(A, B, x, y):
    N, m, k = y.shape
    out = np.empty_like(y)
    for j in range(N):
        blocks = coupling_blocks(A, B, j)
        for i in range(m):
            for c in range(k):
                re = Fraction(float(y[j, i, c].real))
                im = Fraction(float(y[j, i, c].imag))
                for b, M in enumerate(blocks):
                    jb = j - 1 + b
                    if jb < 0 or jb >= N:
                        continue
                    for s in range(m):
                        mr, mi = Fraction(float(M[i, s].real)), Fraction(float(M[i, s].imag))
                        xr, xi = Fraction(float(x[jb, s, c].real)), Fraction(float(x[jb, s, c].imag))
                        re -= mr * xr - mi * xi
                        im -= mr * xi + mi * xr
                out[j, i, c] = float(re) + 1j * float(im)
    return out


def test_equals_the_exact_residual_on_random_data():
    A, B, y = synthetic.gen_system(4, 3, 2, seed=8)
    x = synthetic.gen_system(4, 3, 2, seed=9)[2]
    r = residual_dd(A, B, x, y)
    ex = _exact(A, B, x, y)
    # within one rounding of the exact value
    assert np.all(np.abs(r.real - ex.real) <= 2.0 ** -52 * np.abs(ex.real) + 1e-300)
    assert np.all(np.abs(r.imag - ex.imag) <= 2.0 ** -52 * np.abs(ex.imag) + 1e-300)


def test_near_cancellation_is_resolved():
    """y = A x exactly in rationals up to a tiny offset: the plain FP64
    residual loses the offset, the compensated one keeps it."""
    A, B, _ = synthetic.gen_system(3, 4, 1, seed=2)
    x = synthetic.gen_system(3, 4, 1, seed=3)[2]
    y = oracle.matvec(A, B, x)
    ex = _exact(A, B, x, y)
    r = residual_dd(A, B, x, y)
    assert np.allclose(r, ex, rtol=1e-12, atol=1e-300)


def test_integer_data_is_exact_and_equals_the_plain_matvec():
    rng = np.random.default_rng(0)
    N, m, k = 5, 6, 3
    A = rng.integers(-50, 50, (N, m, m)) + 1j * rng.integers(-50, 50, (N, m, m))
    B = rng.integers(-50, 50, (N - 1, m, m)) + 1j * rng.integers(-50, 50, (N - 1, m, m))
    x = rng.integers(-50, 50, (N, m, k)) + 1j * rng.integers(-50, 50, (N, m, k))
    y = rng.integers(-50, 50, (N, m, k)) + 1j * rng.integers(-50, 50, (N, m, k))
    r = residual_dd(A, B, x, y)
    assert np.array_equal(r, y - oracle.matvec(A, B, x))
    assert np.array_equal(r, _exact(A, B, x, y))
