"""Python binding of the C ABI (include/crsolve.h), same names as the C calls.

PyTorch provides device memory (the plan's workspace and the result tensors)
and streams; every step of the solver runs in libcrsolve's CUDA kernels.
Tensors are complex128 and contiguous:
  A [N, m, m] (lower triangle read), B [N-1, m, m], y and x [N, m, k].
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as nat

__all__ = ["Plan", "crsolve_plan_create", "crsolve_factor", "crsolve_solve", "crsolve_backward",
           "crsolve_info_get", "crsolve_solve_host", "crsolve_plan_levels",
           "crsolve_debug_level_system", "crsolve_timing_enable", "crsolve_timing_read",
           "crsolve_launch_count", "crsolve_mixed_stats", "crsolve_mixed_precondition", "crsolve_tile_set", "crsolve_tile_get", "crsolve_tile_set_mixed", "crsolve_tile_get_mixed",
           "crsolve_solve_noalloc", "crsolve_peak_probe", "crsolve_residual", "solve", "CRSolveFn",
           "NotPositiveDefinite"]


class NotPositiveDefinite(RuntimeError):
    """Raised by the high-level helpers when a Cholesky pivot failed."""

    def __init__(self, info):
        self.info = info
        super().__init__(f"matrix is not positive definite: first breakdown at level {info['level']}, "
                         f"block {info['block']} (original block {info['orig_block']})")


def _vp(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t, shape, name, device=None, cpu=False):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.complex128:
        raise TypeError(f"{name} must be complex128, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if cpu:
        if t.device.type != "cpu":
            raise ValueError(f"{name} must be a host tensor")
    elif t.device.type != "cuda" or (device is not None and t.device != device):
        raise ValueError(f"{name} must live on {device or 'a CUDA device'}")


class Plan:
    """One system shape (N blocks of m x m, right-hand sides up to kmax wide)
    with its device workspace (a torch uint8 tensor owned by this object).

    keep_levels (classic FP64 plans) splits the memory as
    crsolve_plan_keep_levels does: ``workspace`` keeps the factors of levels
    < keep_levels and the level-keep_levels reduced system; ``scratch`` holds
    the coarse levels and the solve buffers.  release_scratch() frees the
    scratch between calls; the next call binds a new one and the solver
    re-factors the coarse levels first (bit-identical results)."""

    def __init__(self, N: int, m: int, kmax: int, precision: int = nat.CRSOLVE_FP64,
                 flags: int = 0, device=None, keep_levels: int | None = None):
        lib = nat.load()
        if not torch.cuda.is_available():
            raise RuntimeError("crsolve needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.N, self.m, self.kmax, self.precision, self.flags = int(N), int(m), int(kmax), int(precision), int(flags)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            nat.check(lib.crsolve_plan_create(self.N, self.m, self.kmax, self.precision, self.flags,
                                              ctypes.byref(self._h)), "crsolve_plan_create")
            self.keep_levels = None if keep_levels is None else int(keep_levels)
            if self.keep_levels is not None:
                nat.check(lib.crsolve_plan_keep_levels(self._h, self.keep_levels), "crsolve_plan_keep_levels")
            nbytes = ctypes.c_size_t()
            nat.check(lib.crsolve_workspace_bytes(self._h, ctypes.byref(nbytes)), "crsolve_workspace_bytes")
            self.workspace_bytes = int(nbytes.value)
            self.workspace = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=self.device)
            nat.check(lib.crsolve_set_workspace(self._h, _vp(self.workspace), self.workspace.numel()),
                      "crsolve_set_workspace")
            self.scratch, self.scratch_bytes = None, 0
            if self.keep_levels is not None:
                nat.check(lib.crsolve_scratch_bytes(self._h, ctypes.byref(nbytes)), "crsolve_scratch_bytes")
                self.scratch_bytes = int(nbytes.value)
                self.ensure_scratch()

    @property
    def handle(self):
        return self._h

    def ensure_scratch(self) -> None:
        """Bind a scratch buffer if this split plan has none (the next solve
        then re-factors the coarse levels)."""
        if self.keep_levels is None or self.scratch is not None:
            return
        with torch.cuda.device(self.device):
            self.scratch = torch.empty(max(self.scratch_bytes, 256), dtype=torch.uint8, device=self.device)
            nat.check(nat.load().crsolve_set_scratch(self._h, _vp(self.scratch), self.scratch.numel()),
                      "crsolve_set_scratch")

    def release_scratch(self) -> None:
        """Unbind and free the scratch of a split plan (call on the stream that
        used it); the workspace alone stays held."""
        if self.keep_levels is None or self.scratch is None:
            return
        nat.check(nat.load().crsolve_set_scratch(self._h, None, 0), "crsolve_set_scratch")
        self.scratch = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            nat.load().crsolve_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def crsolve_plan_create(N, m, kmax, precision=nat.CRSOLVE_FP64, flags=0, device=None) -> Plan:
    return Plan(N, m, kmax, precision, flags, device)


def crsolve_factor(plan: Plan, A: torch.Tensor, B: torch.Tensor | None, stream=None) -> None:
    N, m = plan.N, plan.m
    _need(A, (N, m, m), "A", plan.device)
    if N > 1:
        _need(B, (N - 1, m, m), "B", plan.device)
    plan.ensure_scratch()
    with torch.cuda.device(plan.device):
        nat.check(nat.load().crsolve_factor(plan.handle, _vp(A), _vp(B) if N > 1 else None, _stream(stream)),
                  "crsolve_factor")


def crsolve_solve(plan: Plan, y: torch.Tensor, x: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    N, m = plan.N, plan.m
    k = y.shape[-1] if y.dim() == 3 else -1
    _need(y, (N, m, k), "y", plan.device)
    if x is None:
        x = torch.empty_like(y)
    _need(x, (N, m, k), "x", plan.device)
    plan.ensure_scratch()
    with torch.cuda.device(plan.device):
        nat.check(nat.load().crsolve_solve(plan.handle, k, _vp(y), _vp(x), _stream(stream)), "crsolve_solve")
    return x


def crsolve_mixed_precondition(plan: Plan, r: torch.Tensor, z: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """z = A~^{-1} r with the FP32 factorisation of a factored CRSOLVE_MIXED plan
    (no refinement); r, z: [N, m, k] complex128 on the plan's device."""
    N, m = plan.N, plan.m
    k = r.shape[-1] if r.dim() == 3 else -1
    _need(r, (N, m, k), "r", plan.device)
    if z is None:
        z = torch.empty_like(r)
    _need(z, (N, m, k), "z", plan.device)
    plan.ensure_scratch()
    with torch.cuda.device(plan.device):
        nat.check(nat.load().crsolve_mixed_precondition(plan.handle, k, _vp(r), _vp(z), _stream(stream)),
                  "crsolve_mixed_precondition")
    return z


def crsolve_backward(plan: Plan, x: torch.Tensor, gx: torch.Tensor, want_gA: bool = True,
                     want_gB: bool = True, stream=None):
    N, m = plan.N, plan.m
    k = x.shape[-1]
    _need(x, (N, m, k), "x", plan.device)
    _need(gx, (N, m, k), "gx", plan.device)
    gy = torch.empty_like(gx)
    gA = torch.empty((N, m, m), dtype=torch.complex128, device=plan.device) if want_gA else None
    gB = torch.empty((N - 1, m, m), dtype=torch.complex128, device=plan.device) if (want_gB and N > 1) else None
    plan.ensure_scratch()
    with torch.cuda.device(plan.device):
        nat.check(nat.load().crsolve_backward(plan.handle, k, _vp(x), _vp(gx), _vp(gy), _vp(gA), _vp(gB),
                                              _stream(stream)), "crsolve_backward")
    return gy, gA, gB


def crsolve_info_get(plan: Plan, stream=None) -> dict:
    info = nat.CrsolveInfo()
    with torch.cuda.device(plan.device):
        nat.check(nat.load().crsolve_info_get(plan.handle, ctypes.byref(info), _stream(stream)),
                  "crsolve_info_get")
    return {"status": info.status, "level": info.level, "block": info.block, "orig_block": info.orig_block}


def crsolve_solve_host(plan: Plan, A: torch.Tensor, B: torch.Tensor | None, y: torch.Tensor,
                       x: torch.Tensor | None = None, stream=None):
    """Host tensors in and out (pinned for full copy speed).  Returns (x, status)."""
    N, m = plan.N, plan.m
    k = y.shape[-1]
    _need(A, (N, m, m), "A", cpu=True)
    if N > 1:
        _need(B, (N - 1, m, m), "B", cpu=True)
    _need(y, (N, m, k), "y", cpu=True)
    if x is None:
        x = torch.empty_like(y, pin_memory=y.is_pinned())
    _need(x, (N, m, k), "x", cpu=True)
    plan.ensure_scratch()
    with torch.cuda.device(plan.device):
        rc = nat.check(nat.load().crsolve_solve_host(plan.handle, k, _vp(A), _vp(B) if N > 1 else None,
                                                     _vp(y), _vp(x), _stream(stream)), "crsolve_solve_host")
    return x, rc


def crsolve_plan_levels(plan: Plan):
    lib = nat.load()
    n = ctypes.c_int32()
    nat.check(lib.crsolve_plan_levels(plan.handle, ctypes.byref(n), None), "crsolve_plan_levels")
    sizes = (ctypes.c_int64 * n.value)()
    nat.check(lib.crsolve_plan_levels(plan.handle, ctypes.byref(n), sizes), "crsolve_plan_levels")
    return [int(s) for s in sizes]


def crsolve_debug_level_system(plan: Plan, level: int):
    """Copies of the reduced system (A^(l), B^(l)) of a level >= 1 (tests only)."""
    pa, pb = ctypes.c_void_p(), ctypes.c_void_p()
    nat.check(nat.load().crsolve_debug_level_system(plan.handle, int(level), ctypes.byref(pa), ctypes.byref(pb)),
              "crsolve_debug_level_system")
    sizes = crsolve_plan_levels(plan)
    Nl, m = sizes[level], plan.m
    base = plan.workspace.data_ptr()
    ws = plan.workspace.view(torch.uint8)
    a0, b0 = pa.value - base, pb.value - base
    A = ws[a0:a0 + Nl * m * m * 16].view(torch.complex128).reshape(Nl, m, m).clone()
    B = ws[b0:b0 + max(Nl - 1, 0) * m * m * 16].view(torch.complex128).reshape(max(Nl - 1, 0), m, m).clone()
    return A, B


def crsolve_timing_enable(plan: Plan, enable: bool = True) -> None:
    nat.check(nat.load().crsolve_timing_enable(plan.handle, 1 if enable else 0), "crsolve_timing_enable")


def crsolve_timing_read(plan: Plan, cap: int = 1 << 16):
    """Per-kernel records [(kind, level, units, ms)] since the last read."""
    buf = (nat.CrsolveKernelTime * cap)()
    n = ctypes.c_int32()
    nat.check(nat.load().crsolve_timing_read(plan.handle, buf, cap, ctypes.byref(n)), "crsolve_timing_read")
    return [(nat.KERNEL_KINDS[buf[i].kind], buf[i].level, buf[i].units, buf[i].ms) for i in range(min(n.value, cap))]


def crsolve_mixed_stats(plan: Plan) -> dict:
    it, fb = ctypes.c_int32(), ctypes.c_int32()
    dl, rho = ctypes.c_double(), ctypes.c_double()
    nat.check(nat.load().crsolve_mixed_stats(plan.handle, ctypes.byref(it), ctypes.byref(dl), ctypes.byref(rho),
                                             ctypes.byref(fb)), "crsolve_mixed_stats")
    return {"iterations": int(it.value), "delta": float(dl.value), "rho": float(rho.value),
            "fp64_fallback": bool(fb.value)}


def crsolve_launch_count(plan: Plan) -> int:
    c = ctypes.c_int64()
    nat.check(nat.load().crsolve_launch_count(plan.handle, ctypes.byref(c)), "crsolve_launch_count")
    return int(c.value)


def crsolve_residual(A: torch.Tensor, B: torch.Tensor | None, x: torch.Tensor, y: torch.Tensor,
                     method: str = "split", r: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """r = y - A x for the block-tridiagonal system (method "fp64", "split":
    exact slice products on the tensor cores, or "split_image": the same with
    the matrix slices precomputed in the workspace)."""
    N, m, _ = A.shape
    k = x.shape[-1]
    _need(A, (N, m, m), "A")
    if N > 1:
        _need(B, (N - 1, m, m), "B", A.device)
    _need(x, (N, m, k), "x", A.device)
    _need(y, (N, m, k), "y", A.device)
    if r is None:
        r = torch.empty_like(y)
    code = {"fp64": nat.CRSOLVE_RESIDUAL_FP64, "split": nat.CRSOLVE_RESIDUAL_SPLIT,
            "split_image": nat.CRSOLVE_RESIDUAL_SPLIT_IMAGE}[method]
    lib = nat.load()
    nbytes = ctypes.c_size_t()
    nat.check(lib.crsolve_residual_workspace_bytes(N, m, k, code, ctypes.byref(nbytes)),
              "crsolve_residual_workspace_bytes")
    ws = torch.empty(max(int(nbytes.value), 1), dtype=torch.uint8, device=A.device)
    with torch.cuda.device(A.device):
        nat.check(lib.crsolve_residual(N, m, k, _vp(A), _vp(B) if N > 1 else None, _vp(x), _vp(y), _vp(r), code,
                                       _vp(ws), int(nbytes.value), _stream(stream)), "crsolve_residual")
    return r


def crsolve_peak_probe(kind: str = "fp64", stream=None) -> dict:
    """Measured FMA rate of the current device ("fp64" or "fp32"):
    {"gflops", "fma_per_clk_sm", "sm_mhz"}."""
    code = {"fp64": nat.CRSOLVE_PROBE_FP64_FMA, "fp32": nat.CRSOLVE_PROBE_FP32_FMA}[kind]
    v, c, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    nat.check(nat.load().crsolve_peak_probe(code, ctypes.byref(v), ctypes.byref(c), ctypes.byref(f), _stream(stream)),
              "crsolve_peak_probe")
    return {"gflops": float(v.value), "fma_per_clk_sm": float(c.value), "sm_mhz": float(f.value)}


def crsolve_tile_set(mt: int, nb_factor: int, nb_solve: int, kc: int, threads: int,
                     threads_solve: int | None = None) -> None:
    nat.check(nat.load().crsolve_tile_set(mt, nb_factor, nb_solve, kc, threads,
                                          threads if threads_solve is None else threads_solve), "crsolve_tile_set")


def crsolve_tile_set_mixed(mt: int, nb_factor: int, nb_solve: int, kc: int, threads: int,
                           threads_solve: int | None = None) -> None:
    nat.check(nat.load().crsolve_tile_set_mixed(mt, nb_factor, nb_solve, kc, threads,
                                                threads if threads_solve is None else threads_solve),
              "crsolve_tile_set_mixed")


def crsolve_tile_get_mixed(mt: int):
    v = [ctypes.c_int32() for _ in range(5)]
    nat.check(nat.load().crsolve_tile_get_mixed(mt, *[ctypes.byref(x) for x in v]), "crsolve_tile_get_mixed")
    return tuple(int(x.value) for x in v)


def crsolve_tile_get(mt: int):
    v = [ctypes.c_int32() for _ in range(5)]
    nat.check(nat.load().crsolve_tile_get(mt, *[ctypes.byref(x) for x in v]), "crsolve_tile_get")
    return tuple(int(x.value) for x in v)


def crsolve_solve_noalloc(A: torch.Tensor, B: torch.Tensor | None, y: torch.Tensor,
                          x: torch.Tensor | None = None, want_info: bool = True, stream=None):
    """Factor + solve without any device allocation by the library (its
    intermediates live in a fixed 32 MiB device array; see include/crsolve.h).
    Returns (x, info dict or None)."""
    N, m, _ = A.shape
    k = y.shape[-1]
    _need(A, (N, m, m), "A")
    if N > 1:
        _need(B, (N - 1, m, m), "B", A.device)
    _need(y, (N, m, k), "y", A.device)
    if x is None:
        x = torch.empty_like(y)
    _need(x, (N, m, k), "x", A.device)
    info = nat.CrsolveInfo() if want_info else None
    with torch.cuda.device(A.device):
        nat.check(nat.load().crsolve_solve_noalloc(N, m, k, _vp(A), _vp(B) if N > 1 else None, _vp(y), _vp(x),
                                                   ctypes.byref(info) if want_info else None, _stream(stream)),
                  "crsolve_solve_noalloc")
    if not want_info:
        return x, None
    return x, {"status": info.status, "level": info.level, "block": info.block, "orig_block": info.orig_block}


_METHOD_FLAGS = {"classic": 0, "alg1": nat.CRSOLVE_PLAN_ALG1}


def _method_flags(method: str) -> int:
    try:
        return _METHOD_FLAGS[method]
    except KeyError:
        raise ValueError(f"method must be one of {sorted(_METHOD_FLAGS)}") from None


def solve(A: torch.Tensor, B: torch.Tensor | None, y: torch.Tensor, check: bool = True,
          method: str = "classic", device=None) -> torch.Tensor:
    """x = A^{-1} y for one system.  CUDA tensors are solved on their device;
    host tensors go through crsolve_solve_host on `device` (default: the
    current CUDA device), whose copies overlap the kernels, and x comes back
    as a host tensor (pin the inputs for full copy speed).  method:
    "classic" (classic cyclic reduction, any N) or "alg1" (the paper's
    Algorithm 1, both halves reduced, N a power of two)."""
    N, m, _ = A.shape
    if A.device.type == "cpu":
        A, y = A.contiguous(), y.contiguous()
        B = None if B is None else B.contiguous()
        plan = Plan(N, m, y.shape[-1], flags=_method_flags(method) | nat.CRSOLVE_PLAN_HOST_STAGING, device=device)
        x, rc = crsolve_solve_host(plan, A, B, y)
        if check and rc != 0:
            raise NotPositiveDefinite(crsolve_info_get(plan))
        return x
    plan = Plan(N, m, y.shape[-1], flags=_method_flags(method), device=A.device)
    crsolve_factor(plan, A, B)
    x = crsolve_solve(plan, y)
    if check:
        info = crsolve_info_get(plan)
        if info["status"] != 0:
            raise NotPositiveDefinite(info)
    return x


class CRSolveFn(torch.autograd.Function):
    """x = A^{-1} y with the cyclic-reduction solver; backward by
    crsolve_backward (a Hermitian re-solve with the stored factors and fused
    outer products).  A_j is treated as Hermitian: its gradient is projected
    onto Hermitian matrices.

    keep_factors trades compute for memory between the forward and the
    backward pass:
      True   keep the factors of every level (no recomputation);
      l >= 1 (classic method) keep the factors of the fine levels 0 .. l-1
             and the level-l reduced system, about 1 - 2^-l of the factor
             memory; the backward pass re-factors the coarse levels l .. L
             (about 2^-l of the factorisation);
      False  keep only A, B and x; the backward pass re-factors everything.
    The re-factorisation is deterministic, so the gradients are identical.
    method selects the solver as in ``solve``."""

    @staticmethod
    def forward(ctx, A, B, y, keep_factors=True, method: str = "classic"):
        N, m, _ = A.shape
        A, B, y = A.contiguous(), None if B is None else B.contiguous(), y.contiguous()
        ctx.flags = _method_flags(method)
        if keep_factors is True:
            keep = None
        elif keep_factors is False:
            keep = 0
        else:
            keep = int(keep_factors)
            if keep < 0:
                raise ValueError("keep_factors must be True, False or a level count >= 0")
        if keep is not None and ctx.flags & nat.CRSOLVE_PLAN_ALG1 and keep > 0:
            raise ValueError("keep_factors = l > 0 needs the classic method")
        split = keep is not None and not ctx.flags & nat.CRSOLVE_PLAN_ALG1
        plan = Plan(N, m, y.shape[-1], flags=ctx.flags, device=A.device, keep_levels=keep if split else None)
        crsolve_factor(plan, A, B)
        x = crsolve_solve(plan, y)
        ctx.has_B = B is not None
        ctx.keep = keep
        if keep is None:
            ctx.plan = plan
            ctx.save_for_backward(x)
        elif split:
            # the coarse levels go with the scratch; keep = 0 re-factors from
            # A and B, which the plan reads again in the backward pass
            plan.release_scratch()
            ctx.plan = plan
            ctx.save_for_backward(x, A, B if B is not None else A.new_empty(0))
        else:
            plan.close()
            del plan
            ctx.plan = None
            ctx.save_for_backward(x, A, B if B is not None else A.new_empty(0))
        return x

    @staticmethod
    def backward(ctx, gx):
        if ctx.keep is None:
            (x,) = ctx.saved_tensors
            plan = ctx.plan
        elif ctx.plan is not None:
            x = ctx.saved_tensors[0]
            plan = ctx.plan
        else:
            x, A, B = ctx.saved_tensors
            N, m, _ = A.shape
            plan = Plan(N, m, x.shape[-1], flags=ctx.flags, device=A.device)
            crsolve_factor(plan, A, B if ctx.has_B else None)
        gy, gA, gB = crsolve_backward(plan, x, gx.contiguous(), ctx.needs_input_grad[0],
                                      ctx.needs_input_grad[1] and ctx.has_B)
        return gA, gB, gy if ctx.needs_input_grad[2] else None, None, None
