"""Binding of the batched C ABI: many independent systems of uneven N, m and
k solved by one persistent kernel launch (optionally replayed as a CUDA
graph).  Same names as the C calls; argument marshalling only.

Packed layout (include/crsolve.h): system i's blocks are contiguous and the
systems follow each other in order, so A is one complex128 vector of
sum N_i m_i^2 elements, B of sum (N_i - 1) m_i^2, y and x of sum N_i m_i k_i.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as nat
from .api import _stream, _vp

__all__ = ["Batch", "crsolve_batch_create", "crsolve_batch_solve", "crsolve_batch_graph_launch",
           "crsolve_batch_info"]


class Batch:
    """nsys independent systems; owns its device workspace (a torch tensor).

    tiles: optional {mt: (nb_factor, nb_solve, kc)} per block-size class.
    max_workspace_bytes: cap on the workspace (0 = one slot per resident CTA).
    """

    def __init__(self, Ns, ms, ks, device=None, tiles=None, max_workspace_bytes: int = 0):
        lib = nat.load()
        if not torch.cuda.is_available():
            raise RuntimeError("crsolve needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.Ns = np.ascontiguousarray(Ns, dtype=np.int64)
        self.ms = np.ascontiguousarray(ms, dtype=np.int32)
        self.ks = np.ascontiguousarray(ks, dtype=np.int32)
        if isinstance(tiles, str):
            if tiles != "auto":
                raise ValueError("tiles must be None, 'auto' or {mt: (nb_factor, nb_solve, kc)}")
            from .autotune import tiles_for
            tiles = tiles_for(self.ms, self.ks, self.device)
        self.tiles = dict(tiles or {})
        self.nsys = len(self.Ns)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            nat.check(lib.crsolve_batch_create(self.nsys, self.Ns.ctypes.data_as(ctypes.c_void_p),
                                               self.ms.ctypes.data_as(ctypes.c_void_p),
                                               self.ks.ctypes.data_as(ctypes.c_void_p), ctypes.byref(self._h)),
                      "crsolve_batch_create")
            for mt, (nbf, nbs, kc) in (tiles or {}).items():
                nat.check(lib.crsolve_batch_tile_set(self._h, int(mt), int(nbf), int(nbs), int(kc)),
                          "crsolve_batch_tile_set")
            nbytes, nslots = ctypes.c_size_t(), ctypes.c_int32()
            nat.check(lib.crsolve_batch_workspace_bytes(self._h, int(max_workspace_bytes), ctypes.byref(nbytes),
                                                        ctypes.byref(nslots)), "crsolve_batch_workspace_bytes")
            self.nslots = int(nslots.value)
            self.workspace_bytes = int(nbytes.value)
            self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
            nat.check(lib.crsolve_batch_set_workspace(self._h, _vp(self.workspace), self.workspace.numel()),
                      "crsolve_batch_set_workspace")
        self.offA = np.zeros(self.nsys, np.int64)
        self.offB = np.zeros(self.nsys, np.int64)
        self.offY = np.zeros(self.nsys, np.int64)
        tot = np.zeros(3, np.int64)
        nat.check(lib.crsolve_batch_offsets(self._h, self.offA.ctypes.data_as(ctypes.c_void_p),
                                            self.offB.ctypes.data_as(ctypes.c_void_p),
                                            self.offY.ctypes.data_as(ctypes.c_void_p),
                                            tot.ctypes.data_as(ctypes.c_void_p)), "crsolve_batch_offsets")
        self.nA, self.nB, self.nY = (int(v) for v in tot)

    @property
    def handle(self):
        return self._h

    # packing helpers (host side, for tests and examples)
    def pack(self, systems, device=None):
        """[(A_i, B_i, y_i)] numpy -> packed complex128 tensors on the device."""
        A = np.empty(self.nA, np.complex128)
        B = np.empty(max(self.nB, 1), np.complex128)
        y = np.empty(self.nY, np.complex128)
        for i, (a, b, yy) in enumerate(systems):
            A[self.offA[i]:self.offA[i] + a.size] = a.ravel()
            if b.size:
                B[self.offB[i]:self.offB[i] + b.size] = b.ravel()
            y[self.offY[i]:self.offY[i] + yy.size] = yy.ravel()
        dev = device or self.device
        return (torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev), torch.from_numpy(y).to(dev))

    def system_view(self, i, A, B, y_or_x):
        """Views (A_i [N,m,m], B_i [N-1,m,m], y_i or x_i [N,m,k]) into packed tensors."""
        N, m, k = int(self.Ns[i]), int(self.ms[i]), int(self.ks[i])
        a = A[self.offA[i]:self.offA[i] + N * m * m].view(N, m, m)
        b = B[self.offB[i]:self.offB[i] + (N - 1) * m * m].view(N - 1, m, m)
        v = y_or_x[self.offY[i]:self.offY[i] + N * m * k].view(N, m, k)
        return a, b, v

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            nat.load().crsolve_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def crsolve_batch_create(Ns, ms, ks, device=None, tiles=None, max_workspace_bytes=0) -> Batch:
    return Batch(Ns, ms, ks, device, tiles, max_workspace_bytes)


def _check_packed(b: Batch, A, B, y, x):
    for t, n, name in ((A, b.nA, "A"), (y, b.nY, "y"), (x, b.nY, "x")):
        if t.dtype != torch.complex128 or t.device != b.device or not t.is_contiguous() or t.numel() < n:
            raise ValueError(f"{name} must be a contiguous complex128 tensor of >= {n} elements on {b.device}")
    if b.nB and (B is None or B.dtype != torch.complex128 or B.numel() < b.nB or not B.is_contiguous()):
        raise ValueError(f"B must be a contiguous complex128 tensor of >= {b.nB} elements")


def crsolve_batch_solve(b: Batch, A, B, y, x=None, stream=None):
    if x is None:
        x = torch.empty_like(y)
    _check_packed(b, A, B, y, x)
    with torch.cuda.device(b.device):
        nat.check(nat.load().crsolve_batch_solve(b.handle, _vp(A), _vp(B), _vp(y), _vp(x), _stream(stream)),
                  "crsolve_batch_solve")
    return x


def crsolve_batch_graph_launch(b: Batch, A, B, y, x, stream=None):
    _check_packed(b, A, B, y, x)
    with torch.cuda.device(b.device):
        nat.check(nat.load().crsolve_batch_graph_launch(b.handle, _vp(A), _vp(B), _vp(y), _vp(x),
                                                        _stream(stream)), "crsolve_batch_graph_launch")
    return x


def crsolve_batch_info(b: Batch, stream=None):
    arr = (nat.CrsolveInfo * b.nsys)()
    with torch.cuda.device(b.device):
        nat.check(nat.load().crsolve_batch_info(b.handle, arr, _stream(stream)), "crsolve_batch_info")
    return [{"status": r.status, "level": r.level, "block": r.block, "orig_block": r.orig_block} for r in arr]
