"""Diagonal shifts that give the generator a target condition number.

For A(s) = A0 + s*I, with A0 the generator's system at shift 0 (block
diagonally dominant, hence positive semi-definite), kappa(s) =
(lmax0 + s) / (lmin0 + s), so s = (lmax0 - kappa*lmin0) / (kappa - 1).
lmax0 and lmin0 are computed with ARPACK on the assembled banded Hermitian
matrix (lmin0 by shift-invert through LAPACK's banded Cholesky).  No cyclic
reduction and no GPU is involved; the resulting shifts are inputs of the
kappa-controlled workloads, and kappa is an estimate ("about kappa").

    python tests/golden/make_kappa_shifts.py   # rewrites kappa_shifts.json
"""
import json
import os
import sys

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import synthetic  # noqa: E402

CASES = [  # (name, N, m, k, seed, kappas)
    ("mixed_N2p10_m64_k32", 1 << 10, 64, 32, 4000, [1e2, 1e4, 1e6]),
    ("mixed_N2p14_m64_k32", 1 << 14, 64, 32, 4000, [1e2, 1e4, 1e6]),
    ("plain_N2p12_m8_k4", 1 << 12, 8, 4, 1001, [1e6]),
    ("plain_N2p20_m8_k4", 1 << 20, 8, 4, 1001, [1e6]),
]


def _herm_blocks(A):
    N, m, _ = A.shape
    L = np.tril(A, -1)
    H = L + np.conj(np.swapaxes(L, 1, 2))
    idx = np.arange(m)
    H[:, idx, idx] = A[:, idx, idx].real
    return H


def banded_upper(A, B):
    """LAPACK upper banded storage (bandwidth 2m-1) of the Hermitian matrix of eq. Axb."""
    N, m, _ = A.shape
    n, u = N * m, 2 * m - 1
    ab = np.zeros((u + 1, n), np.complex128)
    H = _herm_blocks(A)
    r, c = np.triu_indices(m)                    # upper part of each diagonal block
    j = np.arange(N)[:, None]
    ab[(u + r - c)[None, :].repeat(N, 0), j * m + c[None, :]] = H[:, r, c]
    if N > 1:
        r2, c2 = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
        r2, c2 = r2.ravel(), c2.ravel()
        j2 = np.arange(N - 1)[:, None]           # block (j, j+1) is B_j^H: entry (r, c) = conj(B_j[c, r])
        ab[(u + r2 - m - c2)[None, :].repeat(N - 1, 0), (j2 + 1) * m + c2[None, :]] = np.conj(B[:, c2, r2])
    return ab


def sparse_of(A, B):
    N, m, _ = A.shape
    H = _herm_blocks(A)
    rr, cc = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    j = np.arange(N)[:, None, None]
    rows = [(j * m + rr).ravel()]
    cols = [(j * m + cc).ravel()]
    vals = [H.ravel()]
    if N > 1:
        j1 = np.arange(N - 1)[:, None, None]
        rows += [((j1 + 1) * m + rr).ravel(), (j1 * m + rr).ravel()]
        cols += [(j1 * m + cc).ravel(), ((j1 + 1) * m + cc).ravel()]
        vals += [B.ravel(), np.conj(np.swapaxes(B, 1, 2)).ravel()]
    n = N * m
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def extremes(A, B):
    S = sparse_of(A, B)
    n = S.shape[0]
    lmax = float(spla.eigsh(S, k=1, which="LA", return_eigenvectors=False, tol=1e-10)[0])
    sigma = -1e-3 * lmax                                 # A0 - sigma*I is positive definite
    ab = banded_upper(A, B)
    ab[-1] -= sigma
    cb = sla.cholesky_banded(ab, lower=False)
    op = spla.LinearOperator((n, n), matvec=lambda v: sla.cho_solve_banded((cb, False), v), dtype=np.complex128)
    mu = float(spla.eigsh(op, k=1, which="LA", return_eigenvectors=False, tol=1e-10)[0])
    return lmax, sigma + 1.0 / mu


def main():
    out = {}
    for name, N, m, k, seed, kappas in CASES:
        A0, B, _ = synthetic.gen_system(N, m, k, seed, shift=0.0)
        lmax0, lmin0 = extremes(A0, B)
        out[name] = {"N": N, "m": m, "k": k, "seed": seed, "lmax0": lmax0, "lmin0": lmin0,
                     "shifts": {f"{kap:.0e}": (lmax0 - kap * lmin0) / (kap - 1.0) for kap in kappas}}
        print(name, out[name], flush=True)
    with open(os.path.join(HERE, "kappa_shifts.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
