"""Dense helpers for pinning the oracle (numpy / LAPACK only; no cyclic reduction)."""
import numpy as np


def herm_from_lower(Aj):
    """The Hermitian matrix that a lower-triangle reader sees in Aj."""
    L = np.tril(Aj, -1)
    return L + L.conj().T + np.diag(np.diag(Aj).real)


def assemble(A, B):
    """Dense matrix of eq. Axb: A_j on the diagonal, B_j at (j+1, j), B_j^H at (j, j+1)."""
    N, m, _ = A.shape
    D = np.zeros((N * m, N * m), dtype=np.complex128)
    for j in range(N):
        D[j * m:(j + 1) * m, j * m:(j + 1) * m] = herm_from_lower(A[j])
        if j + 1 < N:
            D[(j + 1) * m:(j + 2) * m, j * m:(j + 1) * m] = B[j]
            D[j * m:(j + 1) * m, (j + 1) * m:(j + 2) * m] = B[j].conj().T
    return D


def dense_solve(A, B, y):
    N, m, k = y.shape
    return np.linalg.solve(assemble(A, B), y.reshape(N * m, k)).reshape(N, m, k)


def rel_err(x, ref):
    return np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel())


def eta_inf(A, B, x, y):
    """max over rhs columns of ||y - A x||_inf / (||A||_inf ||x||_inf), dense."""
    N, m, k = y.shape
    D = assemble(A, B)
    X = x.reshape(N * m, k)
    R = y.reshape(N * m, k) - D @ X
    nA = np.abs(D).sum(axis=1).max()
    return max(np.abs(R[:, c]).max() / (nA * np.abs(X[:, c]).max()) for c in range(k))
