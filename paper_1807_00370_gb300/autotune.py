"""Tile autotuner of the batched form and of the single-system plans.

Batched form: for every block-size class MT (4, 8, 16, 32, 64) present in a
batch, it times the persistent batched kernel on a sample batch of that class
and keeps the fastest (odd blocks per chunk in the factor step, odd blocks
per chunk in the solve steps, right-hand-side columns per chunk).  Plans
(plan_tiles): per class, width k and precision, a coordinate search over the
five parameters of the plan kernels' tile table.  Results are cached per GPU
name in _build/tiles.json next to the library.  The sample inputs come from
torch's generator (their values do not matter for timing, only their shapes;
they are diagonally dominant, so every sample factorises).
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import build as _build
from .batched import Batch, crsolve_batch_solve

CACHE = os.path.join(_build.BUILD, "tiles.json")
NB_CANDIDATES = (1, 2, 4, 8, 16, 32)
KC_CANDIDATES = (8, 16, 32)


def _mt(m: int) -> int:
    for c in (4, 8, 16, 32, 64):
        if m <= c:
            return c
    raise ValueError("m > 64")


def _sample_inputs(Ns, ms, ks, device):
    tot_a = int((Ns * ms * ms).sum())
    tot_b = int(((Ns - 1) * ms * ms).sum())
    tot_y = int((Ns * ms * ks).sum())
    g = torch.Generator(device=device).manual_seed(1234)

    def rnd(n):
        return torch.view_as_complex(torch.randn(n, 2, generator=g, device=device, dtype=torch.float64))

    A = rnd(tot_a) * 0.05
    B = rnd(max(tot_b, 1)) * 0.05
    # make every diagonal block strongly diagonal: A_j += (2 + small) I
    off = 0
    for N, m in zip(Ns, ms):
        idx = torch.arange(m, device=device)
        blk = A[off:off + N * m * m].view(N, m, m)
        blk[:, idx, idx] += 4.0
        off += N * m * m
    return A, B, rnd(tot_y)


def _time(b: Batch, A, B, y, x, reps=3) -> float:
    crsolve_batch_solve(b, A, B, y, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        crsolve_batch_solve(b, A, B, y, x)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_class(mt: int, m: int, k: int, device=None, n_blocks: int = 512, verbose: bool = False):
    """Best (nb_factor, nb_solve, kc) for class mt on systems of size m, width k."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    nslots_guess = torch.cuda.get_device_properties(device).multi_processor_count * 2
    nsys = 2 * nslots_guess
    Ns = np.full(nsys, n_blocks, np.int64)
    ms = np.full(nsys, m, np.int32)
    ks = np.full(nsys, k, np.int32)
    A, B, y = _sample_inputs(Ns, ms, ks, device)
    x = torch.empty_like(y)
    best = None

    def trial(nbf, nbs, kc):
        try:
            b = Batch(Ns, ms, ks, device=device, tiles={mt: (nbf, nbs, kc)})
        except RuntimeError:
            return None                      # does not fit in shared memory
        t = _time(b, A, B, y, x)
        if verbose:
            print(f"  mt={mt} nbf={nbf} nbs={nbs} kc={kc}: {t:.3f} ms")
        return t

    # factor chunk first (solve tile at its default), then the solve chunk
    res_f = {}
    for nbf in NB_CANDIDATES:
        t = trial(nbf, 1, min(16, k))
        if t is not None:
            res_f[nbf] = t
    nbf = min(res_f, key=res_f.get)
    res_s = {}
    for nbs in NB_CANDIDATES:
        for kc in KC_CANDIDATES:
            if kc > max(k, 8):
                continue
            t = trial(nbf, nbs, kc)
            if t is not None:
                res_s[(nbs, kc)] = t
    (nbs, kc) = min(res_s, key=res_s.get)
    best = (int(nbf), int(nbs), int(kc))
    return best, {"factor": res_f, "solve": {f"{a},{c}": v for (a, c), v in res_s.items()}}


def load_cache():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tiles_for(ms, ks, device=None, use_cache: bool = True, verbose: bool = False):
    """{mt: (nb_factor, nb_solve, kc)} for the classes present in a batch."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    name = torch.cuda.get_device_name(device)
    cache = load_cache() if use_cache else {}
    out, changed = {}, False
    ms = np.asarray(ms)
    ks = np.asarray(ks)
    for mt in sorted({_mt(int(m)) for m in ms}):
        key = f"{name}|mt={mt}"
        if key not in cache:
            sel = np.array([_mt(int(m)) == mt for m in ms])
            m_rep = int(np.max(ms[sel]))
            k_rep = int(np.median(ks[sel]))
            best, table = tune_class(mt, m_rep, k_rep, device, verbose=verbose)
            cache[key] = {"tile": best, "m": m_rep, "k": k_rep, "timings_ms": table}
            changed = True
        out[mt] = tuple(cache[key]["tile"])
    if changed:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    return out


# ------------------------------------------------- single-system (plan) paths
#
# The plan kernels read a process-wide tile table per block-size class and
# precision (crsolve_tile_set / crsolve_tile_set_mixed).  plan_tiles() picks a
# shape for (class, k, precision) by timing factor + solve of a sample system
# over the candidates (each parameter around the current shape, a coordinate
# search), caches it per GPU name under that key, and with apply=True writes
# it into the table for later launches of every plan of that class.

PLAN_NB = (1, 2, 4, 8, 16, 32)
PLAN_KC = (8, 16, 32)
PLAN_THREADS = (128, 256)


def _time_plan(N, m, k, precision, A, B, y, reps=3) -> float:
    from .api import Plan, crsolve_factor, crsolve_solve
    plan = Plan(N, m, k, precision=precision)
    x = torch.empty_like(y)
    crsolve_factor(plan, A, B)
    crsolve_solve(plan, y, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        crsolve_factor(plan, A, B)
        crsolve_solve(plan, y, x)
    e1.record()
    torch.cuda.synchronize()
    plan.close()
    return e0.elapsed_time(e1) / reps


def tune_plan_class(m: int, k: int, precision: int = 0, n_blocks: int = 0, device=None, verbose: bool = False):
    """Best (nb_factor, nb_solve, kc, threads, threads_solve) of class mt(m)
    for width k and precision (0 FP64, 1 mixed: its FP32 levels' table) on a
    sample system of n_blocks blocks (default: 2^20 / m^2, at least 2^12).
    Restores the table it started from; returns (shape, timings)."""
    from . import api
    device = device or torch.device("cuda", torch.cuda.current_device())
    mt = _mt(m)
    getter = api.crsolve_tile_get_mixed if precision else api.crsolve_tile_get
    setter = api.crsolve_tile_set_mixed if precision else api.crsolve_tile_set
    if n_blocks <= 0:
        n_blocks = max(1 << 12, (1 << 20) // (m * m))
    A, B, y = _sample_inputs(np.array([n_blocks]), np.array([m]), np.array([k]), device)
    A = A.view(n_blocks, m, m)
    B = B[:(n_blocks - 1) * m * m].view(n_blocks - 1, m, m)
    y = y.view(n_blocks, m, k)
    start = list(getter(mt))
    best, timings = list(start), {}

    def trial(shape):
        key = ",".join(map(str, shape))
        if key in timings:
            return timings[key]
        try:
            setter(mt, *shape)
        except Exception:  # noqa: BLE001 - out of range or too large for shared memory
            timings[key] = None
            return None
        t = _time_plan(n_blocks, m, k, precision, A, B, y)
        timings[key] = t
        if verbose:
            print(f"  mt={mt} k={k} prec={precision} {shape}: {t:.3f} ms")
        return t

    # The FP32 levels of class 64 solve with fixed-shape product kernels (one
    # odd block per work item, chunk by k): only the factor fields matter there.
    knobs = (PLAN_NB, PLAN_NB, PLAN_KC, PLAN_THREADS, PLAN_THREADS)
    factor_only = {0, 3}
    try:
        t_best = trial(best)
        for i, cands in enumerate(knobs):
            if precision and mt == 64 and i not in factor_only:
                continue
            for v in cands:
                shape = list(best)
                shape[i] = v
                t = trial(shape)
                if t is not None and t < t_best:
                    best, t_best = shape, t
    finally:
        setter(mt, *start)
    return tuple(int(v) for v in best), {k_: v for k_, v in timings.items() if v is not None}


def plan_tiles(m: int, k: int, precision: int = 0, device=None, use_cache: bool = True, apply: bool = True,
               verbose: bool = False):
    """The tuned tile shape of class mt(m) for width k and precision, from the
    cache (key: GPU name, class, k rounded up to a power of two, precision)
    or tuned now; with apply=True it is written into the process-wide table."""
    from . import api
    device = device or torch.device("cuda", torch.cuda.current_device())
    name = torch.cuda.get_device_name(device)
    kb = 1 << max(0, (int(k) - 1).bit_length())
    key = f"{name}|plan|mt={_mt(m)}|k={kb}|prec={'mixed' if precision else 'fp64'}"
    cache = load_cache() if use_cache else {}
    if key not in cache:
        best, table = tune_plan_class(m, kb, precision, device=device, verbose=verbose)
        cache = load_cache()
        cache[key] = {"tile": list(best), "m": int(m), "k": kb, "timings_ms": table}
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    shape = tuple(cache[key]["tile"])
    if apply:
        (api.crsolve_tile_set_mixed if precision else api.crsolve_tile_set)(_mt(m), *shape)
    return shape
