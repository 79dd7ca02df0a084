"""CPU oracle for classic cyclic reduction (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does.

The arithmetic lives in ``cr_oracle.c`` (plain C99 complex doubles, naive
loops, OpenMP over the blocks of one level only); this module compiles it
with gcc and exposes numpy-friendly wrappers.  Everything is complex128.

Functions and the passages they follow:
  cr_solve     classic cyclic reduction, Sec. 2 (eq. even, eq. Formulas, the
               boundary auxiliaries, the Cholesky base case and the
               breakdown test) with Sec. 4's Cholesky product rule; odd
               unknowns by back-substitution from the odd rows of eq. Axb
  cr_level     one reduction level (eq. Formulas, even half)
  matvec       the block-tridiagonal product of eq. Axb
  cr_backward  adjoint of x = A^{-1} y (the paper has no adjoint; this is the
               plain definition: gy = A^{-1} gx, gA = -herm(gy x^H),
               gB_j = -(gy_{j+1} x_j^H + x_{j+1} gy_j^H))
  alg1_solve   the paper's own recursion, Algorithm 1 (Sec. 3): both the odd
               system (U, E, u) and the even system (V, F, v) of eq. Formulas
               are formed and solved recursively down to single blocks
               (N a power of two)
  alg1_split   one split of Algorithm 1 (eq. Formulas, both halves)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libcr_oracle.so")
_lock = threading.Lock()
_lib = None


class OracleInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("level", ctypes.c_int32),
                ("block", ctypes.c_int64), ("orig_block", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile cr_oracle.c into _build/libcr_oracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.abspath(__file__)))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        # C99 complex semantics (no -fcx-limited-range): finite products are
        # the plain formula either way; non-finite ones keep Annex G rules
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        try:
            lib = ctypes.CDLL(_LIB)
        except OSError:
            build(force=True)          # e.g. a library built on another architecture
            lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int
        lib.oracle_cr_solve.argtypes = [i64, i32, i32, P, P, P, P, ctypes.POINTER(OracleInfo)]
        lib.oracle_cr_solve.restype = i32
        lib.oracle_cr_level.argtypes = [i64, i32, i32, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_cr_level.restype = i64
        lib.oracle_cr_backsub.argtypes = [i64, i32, i32, P, P, P, P, P, P]
        lib.oracle_cr_backsub.restype = None
        lib.oracle_matvec.argtypes = [i64, i32, i32, P, P, P, P]
        lib.oracle_matvec.restype = None
        lib.oracle_cr_backward.argtypes = [i64, i32, i32, P, P, P, P, P, P, P]
        lib.oracle_cr_backward.restype = i32
        lib.oracle_alg1_solve.argtypes = [i64, i32, i32, P, P, P, P, ctypes.POINTER(OracleInfo)]
        lib.oracle_alg1_solve.restype = i32
        lib.oracle_alg1_split.argtypes = [i64, i32, i32, P, P, P, P, P, P, P, P, P]
        lib.oracle_alg1_split.restype = i64
        lib.oracle_set_threads.argtypes = [i32]
        lib.oracle_set_threads.restype = None
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = i32
        _lib = lib
        return lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _shapes(A, B, y):
    N, m, m2 = A.shape
    assert m == m2, "A must be [N, m, m]"
    assert B.shape == (max(N - 1, 0), m, m), "B must be [N-1, m, m]"
    if y is not None:
        assert y.shape[:2] == (N, m), "y must be [N, m, k]"
    return N, m


def cr_solve(A, B, y):
    """x = A^{-1} y by classic CR.  Returns (x, info dict)."""
    lib = _load()
    A, B, y = _c(A), _c(B), _c(y)
    N, m = _shapes(A, B, y)
    k = y.shape[2]
    x = np.empty_like(y)
    info = OracleInfo()
    lib.oracle_cr_solve(N, m, k, _p(A), _p(B) if N > 1 else None, _p(y), _p(x), ctypes.byref(info))
    return x, {"status": info.status, "level": info.level, "block": info.block,
               "orig_block": info.orig_block}


def cr_level(A, B, y=None):
    """One reduction level.  Returns a dict with L, P, Q, r (odd blocks),
    An, Bn, yn (the even system) and fail (0 or the first failing 1-based
    local block)."""
    lib = _load()
    A, B = _c(A), _c(B)
    N, m = _shapes(A, B, y)
    no, ne = (N + 1) // 2, N // 2
    k = 1 if y is None else y.shape[2]
    y = None if y is None else _c(y)
    L = np.zeros((no, m, m), np.complex128)
    P = np.zeros_like(L)
    Q = np.zeros_like(L)
    r = np.zeros((no, m, k), np.complex128) if y is not None else None
    An = np.zeros((ne, m, m), np.complex128)
    Bn = np.zeros((max(ne - 1, 0), m, m), np.complex128)
    yn = np.zeros((ne, m, k), np.complex128) if y is not None else None
    fail = lib.oracle_cr_level(N, m, k, _p(A), _p(B) if N > 1 else None, _p(y), _p(L), _p(P), _p(Q),
                               _p(r), _p(An) if ne else None, _p(Bn) if ne > 1 else None,
                               _p(yn) if (ne and y is not None) else None)
    return {"L": L, "P": P, "Q": Q, "r": r, "An": An, "Bn": Bn, "yn": yn, "fail": int(fail)}


def matvec(A, B, x):
    """Block-tridiagonal product A x (A_j Hermitian from its lower triangle)."""
    lib = _load()
    A, B, x = _c(A), _c(B), _c(x)
    N, m = _shapes(A, B, x)
    out = np.empty_like(x)
    lib.oracle_matvec(N, m, x.shape[2], _p(A), _p(B) if N > 1 else None, _p(x), _p(out))
    return out


def cr_backward(A, B, x, gx):
    """Adjoint: returns (gy, gA, gB, status)."""
    lib = _load()
    A, B, x, gx = _c(A), _c(B), _c(x), _c(gx)
    N, m = _shapes(A, B, x)
    gy = np.empty_like(x)
    gA = np.empty_like(A)
    gB = np.empty_like(B)
    st = lib.oracle_cr_backward(N, m, x.shape[2], _p(A), _p(B) if N > 1 else None, _p(x), _p(gx),
                                _p(gy), _p(gA), _p(gB) if N > 1 else None)
    return gy, gA, gB, int(st)


def alg1_solve(A, B, y):
    """x = A^{-1} y by Algorithm 1 (N a power of two).  Returns (x, info dict);
    info["level"] is the recursion depth of the first breakdown and
    info["orig_block"] the smallest failing original block at that depth."""
    lib = _load()
    A, B, y = _c(A), _c(B), _c(y)
    N, m = _shapes(A, B, y)
    if N < 1 or N & (N - 1):
        raise ValueError("Algorithm 1 needs N to be a power of two")
    k = y.shape[2]
    x = np.empty_like(y)
    info = OracleInfo()
    lib.oracle_alg1_solve(N, m, k, _p(A), _p(B) if N > 1 else None, _p(y), _p(x), ctypes.byref(info))
    return x, {"status": info.status, "level": info.level, "block": info.block,
               "orig_block": info.orig_block}


def alg1_split(A, B, y=None):
    """One split of Algorithm 1 on an even number of blocks.  Returns a dict
    with U, E, u (odd system), V, F, v (even system) and fail (0 or the
    smallest failing 1-based block index)."""
    lib = _load()
    A, B = _c(A), _c(B)
    N, m = _shapes(A, B, y)
    if N < 2 or N % 2:
        raise ValueError("a split needs an even number of blocks")
    h = N // 2
    k = 1 if y is None else y.shape[2]
    y = None if y is None else _c(y)
    U = np.zeros((h, m, m), np.complex128)
    V = np.zeros_like(U)
    E = np.zeros((max(h - 1, 0), m, m), np.complex128)
    F = np.zeros_like(E)
    u = np.zeros((h, m, k), np.complex128) if y is not None else None
    v = np.zeros_like(u) if y is not None else None
    fail = lib.oracle_alg1_split(N, m, k, _p(A), _p(B), _p(y), _p(U), _p(E) if h > 1 else None, _p(u),
                                 _p(V), _p(F) if h > 1 else None, _p(v))
    return {"U": U, "E": E, "u": u, "V": V, "F": F, "v": v, "fail": int(fail)}
