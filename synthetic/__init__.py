"""Seeded synthetic workloads for the block-tridiagonal HPD problem (Sec. 1, eq. Axb / eq. Data).

This module only draws random numbers and assembles the input blocks; it
contains none of the cyclic-reduction arithmetic.  Both the CPU oracle tests
and the GPU path take their inputs from here, so that both sides see the same
bytes.

Layout (shared by every consumer):
  A : complex128 [N, m, m]   diagonal blocks A_j (row-major; Hermitian)
  B : complex128 [N-1, m, m] sub-diagonal blocks B_j, sitting at block
                             position (j+1, j); B_j^H sits at (j, j+1)
  y : complex128 [N, m, k]   right-hand-side blocks y_j

Recipe (the paper has no datasets; these shapes follow its problem statement
with m, k << N):
  * B_j = (0.5 / sqrt(m)) * CN(m x m)
  * G_j ~ CN(m x m)
  * A_j = G_j G_j^H / m + (||B_{j-1}||_2 + ||B_j||_2 + s) * I, with
    ||B_0|| = ||B_N|| = 0 and the diagonal shift s = 1 by default.  For
    s > 0 block diagonal dominance gives lambda_min(A) >= s, so the default
    systems have kappa of order 10.  Smaller (or slightly negative) s raises
    kappa; the shifts that give a target kappa are stored in
    tests/golden/kappa_shifts.json by a script that uses only banded LAPACK
    and ARPACK (not cyclic reduction).
  * y_j ~ CN(m x k)
CN(0,1) means re, im ~ N(0, 1/2) independently, so E|z|^2 = 1.
Draw order from numpy's PCG64 ``default_rng(seed)``: B, G, y, then the
optional cotangent c.
"""
from __future__ import annotations

import numpy as np

__all__ = ["cn", "gen_system", "gen_cotangent", "make_indefinite",
           "gen_batch_shapes", "gen_batch", "spectral_norms"]


def cn(rng: np.random.Generator, shape) -> np.ndarray:
    """Complex standard normal CN(0,1): re, im ~ N(0, 1/2)."""
    z = rng.standard_normal(tuple(shape) + (2,))
    return ((z[..., 0] + 1j * z[..., 1]) * np.sqrt(0.5)).astype(np.complex128)


def spectral_norms(B: np.ndarray) -> np.ndarray:
    """||B_j||_2 for every block, via the largest eigenvalue of B_j^H B_j."""
    if B.shape[0] == 0:
        return np.zeros(0)
    out = np.empty(B.shape[0])
    chunk = 1 << 16
    for s in range(0, B.shape[0], chunk):
        b = B[s:s + chunk]
        g = np.conj(np.swapaxes(b, 1, 2)) @ b
        out[s:s + chunk] = np.sqrt(np.maximum(np.linalg.eigvalsh(g)[:, -1], 0.0))
    return out


def gen_system(N: int, m: int, k: int, seed: int, shift: float = 1.0):
    """One HPD block-tridiagonal system with the recipe above.

    Returns (A, B, y) as C-contiguous complex128 arrays.
    """
    if N < 1 or m < 1 or k < 1:
        raise ValueError("N, m, k must be >= 1")
    rng = np.random.default_rng(seed)
    B = cn(rng, (N - 1, m, m)) * (0.5 / np.sqrt(m))
    A = np.empty((N, m, m), dtype=np.complex128)
    chunk = 1 << 16
    for s in range(0, N, chunk):
        G = cn(rng, (min(chunk, N - s), m, m))
        A[s:s + chunk] = G @ np.conj(np.swapaxes(G, 1, 2)) / m
    y = cn(rng, (N, m, k))
    nb = spectral_norms(B)
    dshift = np.full(N, float(shift))
    dshift[1:] += nb          # ||B_{j-1}||
    dshift[:-1] += nb         # ||B_j||
    idx = np.arange(m)
    A[:, idx, idx] += dshift[:, None]
    # exact Hermitian symmetry of the stored diagonal blocks
    A = 0.5 * (A + np.conj(np.swapaxes(A, 1, 2)))
    A[:, idx, idx] = A[:, idx, idx].real
    return np.ascontiguousarray(A), np.ascontiguousarray(B), np.ascontiguousarray(y)


def gen_cotangent(N: int, m: int, k: int, seed: int) -> np.ndarray:
    """The cotangent c of the loss Re sum(conj(c) * x); drawn from its own stream."""
    rng = np.random.default_rng(seed + 7919)
    return cn(rng, (N, m, k))


def make_indefinite(A: np.ndarray, block: int | None = None, amount: float = 3.0) -> np.ndarray:
    """Subtract amount*I from A_block (1-based; default the block N/2)."""
    A = A.copy()
    N, m, _ = A.shape
    j = (N // 2 if block is None else block) - 1
    A[j] -= amount * np.eye(m)
    return A


def gen_batch_shapes(nsys: int, seed: int, n_lo=16, n_hi=4096, ms=(4, 8, 16, 32), k_lo=1, k_hi=16):
    """Uneven batch: N ~ U[n_lo, n_hi], m from ms, k ~ U[k_lo, k_hi] per system."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(n_lo, n_hi + 1, size=nsys)
    mm = rng.choice(np.asarray(ms), size=nsys)
    ks = rng.integers(k_lo, k_hi + 1, size=nsys)
    return Ns.astype(np.int64), mm.astype(np.int32), ks.astype(np.int32)


def gen_batch(Ns, ms, ks, seed: int):
    """List of (A, B, y) for each system; system i uses seed*100003 + i."""
    return [gen_system(int(n), int(m), int(k), seed * 100003 + i)
            for i, (n, m, k) in enumerate(zip(Ns, ms, ks))]


def batch_offsets(Ns, ms, ks):
    """Packed layout of a batch (systems back to back in order): element
    offsets of each system in A, B, y/x and the totals."""
    Ns = np.asarray(Ns, np.int64)
    ms = np.asarray(ms, np.int64)
    ks = np.asarray(ks, np.int64)
    sa, sb, sy = Ns * ms * ms, (Ns - 1) * ms * ms, Ns * ms * ks
    off = lambda s: np.concatenate([[0], np.cumsum(s)[:-1]]).astype(np.int64)
    return off(sa), off(sb), off(sy), (int(sa.sum()), int(sb.sum()), int(sy.sum()))


def gen_batch_device(Ns, ms, ks, seed: int, device="cuda", shift: float = 1.0):
    """The same recipe as gen_system for a whole batch, drawn with torch's
    generator on `device` (fast for batches of ~100 GB) and packed back to
    back (batch_offsets).  Returns packed complex128 tensors (A, B, y)."""
    import torch
    Ns = np.asarray(Ns, np.int64)
    ms = np.asarray(ms, np.int64)
    ks = np.asarray(ks, np.int64)
    offA, offB, offY, (nA, nB, nY) = batch_offsets(Ns, ms, ks)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    A = torch.empty(nA, dtype=torch.complex128, device=device)
    B = torch.empty(max(nB, 1), dtype=torch.complex128, device=device)
    y = torch.empty(nY, dtype=torch.complex128, device=device)

    def cn_t(shape):
        z = torch.randn(tuple(shape) + (2,), generator=gen, device=device, dtype=torch.float64) * np.sqrt(0.5)
        return torch.view_as_complex(z)

    for m in sorted(set(ms.tolist())):
        sel = np.nonzero(ms == m)[0]
        nblk = int(Ns[sel].sum())
        nbb = int((Ns[sel] - 1).sum())
        Bc = cn_t((nbb, m, m)) * (0.5 / np.sqrt(m))
        Gc = cn_t((nblk, m, m))
        Ac = Gc @ Gc.conj().transpose(1, 2) / m
        del Gc
        nb = torch.empty(nbb, dtype=torch.float64, device=device)
        for c0 in range(0, nbb, 16384):          # cuSOLVER's batched eigensolver wants modest batches
            bc = Bc[c0:c0 + 16384]
            nb[c0:c0 + 16384] = torch.sqrt(torch.linalg.eigvalsh(bc.conj().transpose(1, 2) @ bc)[:, -1].clamp_min(0.0))
        # per-block diagonal shift: ||B_{j-1}|| + ||B_j|| + shift, within each system
        dsh = torch.full((nblk,), float(shift), dtype=torch.float64, device=device)
        a0 = b0 = 0
        left_idx, right_idx, nb_idx = [], [], []
        for i in sel:
            N = int(Ns[i])
            if N > 1:
                left_idx.append(np.arange(a0 + 1, a0 + N))     # block j >= 1 gets ||B_{j-1}||
                right_idx.append(np.arange(a0, a0 + N - 1))    # block j <= N-2 gets ||B_j||
                nb_idx.append(np.arange(b0, b0 + N - 1))
            a0 += N
            b0 += N - 1
        if nb_idx:
            li = torch.from_numpy(np.concatenate(left_idx)).to(device)
            ri = torch.from_numpy(np.concatenate(right_idx)).to(device)
            bi = torch.from_numpy(np.concatenate(nb_idx)).to(device)
            dsh.index_add_(0, li, nb[bi])
            dsh.index_add_(0, ri, nb[bi])
        idx = torch.arange(m, device=device)
        Ac[:, idx, idx] += dsh[:, None].to(torch.complex128)
        Ac = 0.5 * (Ac + Ac.conj().transpose(1, 2))
        Ac[:, idx, idx] = Ac[:, idx, idx].real.to(torch.complex128)
        ktot = int((Ns[sel] * m * ks[sel]).sum())
        yc = cn_t((ktot,))
        a0 = b0 = y0 = 0
        for i in sel:
            N, k = int(Ns[i]), int(ks[i])
            A[offA[i]:offA[i] + N * m * m] = Ac[a0:a0 + N].reshape(-1)
            if N > 1:
                B[offB[i]:offB[i] + (N - 1) * m * m] = Bc[b0:b0 + N - 1].reshape(-1)
            y[offY[i]:offY[i] + N * m * k] = yc[y0:y0 + N * m * k]
            a0 += N
            b0 += N - 1
            y0 += N * m * k
        del Ac, Bc, yc
    return A, B, y
