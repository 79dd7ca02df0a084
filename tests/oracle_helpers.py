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


def _split27(a):
    c = 134217729.0 * a          # 2^27 + 1 (Veltkamp)
    hi = c - (c - a)
    return hi, a - hi


def _two_prod(a, b):
    """a * b = p + e exactly (Dekker), elementwise on float64 arrays."""
    p = a * b
    ah, al = _split27(a)
    bh, bl = _split27(b)
    return p, ((ah * bh - p) + ah * bl + al * bh) + al * bl


def _two_sum(a, b):
    """a + b = s + e exactly (Knuth), elementwise."""
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def coupling_blocks(A, B, j):
    """The three complex blocks [B_{j-1} | A_j | B_j^H] of block row j (A_j
    Hermitian from its lower triangle), zero outside the matrix."""
    N, m, _ = A.shape
    z = np.zeros((m, m), np.complex128)
    return (B[j - 1] if j > 0 else z, herm_from_lower(A[j]), B[j].conj().T if j + 1 < N else z)


def residual_dd(A, B, x, y, rows=None):
    """r = y - A x for the listed block rows (default all), every real
    product and sum carried as an unevaluated pair of doubles (Dot2 of Ogita,
    Rump and Oishi): the result is the exact residual rounded, up to a
    relative 2^-104-level error in the sums.  Returns [len(rows)][m][k]."""
    N, m, k = y.shape
    rows = np.arange(N) if rows is None else np.asarray(list(rows))
    R = len(rows)
    Ms, Xs = [], []
    for b in range(3):
        M = np.zeros((R, m, m), np.complex128)
        X = np.zeros((R, m, k), np.complex128)
        for n, j in enumerate(rows):
            M[n] = coupling_blocks(A, B, int(j))[b]
            jb = int(j) - 1 + b
            if 0 <= jb < N:
                X[n] = x[jb]
        Ms.append(M)
        Xs.append(X)
    sr, er = y[rows].real.copy(), np.zeros((R, m, k))
    si, ei = y[rows].imag.copy(), np.zeros((R, m, k))
    for M, X in zip(Ms, Xs):
        for s in range(m):
            mr, mi = M[:, :, s].real[:, :, None], M[:, :, s].imag[:, :, None]
            xr, xi = X[:, s, :].real[:, None, :], X[:, s, :].imag[:, None, :]
            # re: - (mr xr - mi xi); im: - (mr xi + mi xr)
            for (u, v, sg, tgt) in ((mr, xr, -1.0, 0), (mi, xi, 1.0, 0), (mr, xi, -1.0, 1), (mi, xr, -1.0, 1)):
                p, e = _two_prod(np.broadcast_to(u * sg, (R, m, k)), np.broadcast_to(v, (R, m, k)))
                if tgt == 0:
                    sr, e2 = _two_sum(sr, p)
                    er = er + (e + e2)
                else:
                    si, e2 = _two_sum(si, p)
                    ei = ei + (e + e2)
    return (sr + er) + 1j * (si + ei)
