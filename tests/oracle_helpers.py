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


def dense_schur(D, keep, m):
    """Schur complement of the dense matrix D onto the block rows `keep`;
    returns (S, kept scalar rows, eliminated scalar rows)."""
    rows = np.concatenate([np.arange(b * m, (b + 1) * m) for b in keep])
    rest = np.setdiff1d(np.arange(D.shape[0]), rows)
    S = D[np.ix_(rows, rows)]
    if rest.size:
        S = S - D[np.ix_(rows, rest)] @ np.linalg.solve(D[np.ix_(rest, rest)], D[np.ix_(rest, rows)])
    return S, rows, rest


def brute_force_first_failure(A, B, margin):
    """For Algorithm 1 on N = 2^L blocks: the first (depth, 1-based original
    block) whose diagonal block, in the dense Schur complement of the whole
    matrix onto its residue class i = s (mod 2^depth), is not positive
    definite (the split system at that depth that holds those unknowns is
    exactly that Schur complement).  None if every block passes; ValueError
    if some block is within `margin` of singular (too close to call)."""
    N, m, _ = A.shape
    D = assemble(A, B)
    L = N.bit_length() - 1
    for d in range(L + 1):
        fails = []
        for s0 in range(1 << d):
            keep = np.arange(s0, N, 1 << d)
            S, _, _ = dense_schur(D, keep, m)
            for j, b in enumerate(keep):
                lam = np.linalg.eigvalsh(S[j * m:(j + 1) * m, j * m:(j + 1) * m]).min()
                if abs(lam) < margin:
                    raise ValueError("too close to call")
                if lam < 0:
                    fails.append(int(b) + 1)
        if fails:
            return d, min(fails)
    return None


def brute_force_first_failure_classic(A, B, margin):
    """For classic cyclic reduction on any N: the first (level, 1-based local
    odd block) whose diagonal block is not positive definite, found without
    any reduction step.  The level-l system of classic reduction is the dense
    Schur complement of the whole matrix onto the original blocks
    2^l, 2*2^l, ..., N_l*2^l (1-based), so the odd block i of level l is
    diagonal block i of that Schur complement.  At the first level with a
    failure every failing odd block is listed; the smallest is returned as
    (level, block, [all failing blocks]).  None if every block passes;
    ValueError if some block is within `margin` of singular."""
    N, m, _ = A.shape
    D = assemble(A, B)
    level, Nl = 0, N
    while True:
        keep = np.arange(1 << level, N + 1, 1 << level) - 1
        assert len(keep) == Nl
        S, _, _ = dense_schur(D, keep, m)
        fails = []
        for i in range(1, Nl + 1, 2):
            j = i - 1
            lam = np.linalg.eigvalsh(S[j * m:(j + 1) * m, j * m:(j + 1) * m]).min()
            if abs(lam) < margin:
                raise ValueError("too close to call")
            if lam < 0:
                fails.append(i)
        if fails:
            return level, min(fails), fails
        if Nl == 1:
            return None
        Nl //= 2
        level += 1


def shift_blocks(A, blocks, excess=0.5):
    """A copy of A with the Hermitian diagonal blocks at the given 1-based
    original indices shifted by -(lambda_min + excess) I, so that each of them
    is indefinite with lambda_min = -excess."""
    A = A.copy()
    m = A.shape[1]
    for b in blocks:
        lam = np.linalg.eigvalsh(herm_from_lower(A[b - 1])).min()
        A[b - 1] -= (lam + excess) * np.eye(m)
    return A
