"""Small parity cases run on the bounds-checked library (CRSOLVE_LIBRARY=debug,
libcrsolve_debug.so): every result against the oracle, and every plan's and
batch's out-of-range record empty.  Run as a child process by
tests/test_gpu_debug_bounds.py (the library is chosen when it is loaded)."""
import ctypes
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synthetic  # noqa: E402
import paper_1807_00370_gb300 as crs  # noqa: E402
from paper_1807_00370_gb300 import _native as nat  # noqa: E402

NONE = (1 << 64) - 1
TOL = 1e-12


def rel(x, ref):
    return float(np.linalg.norm((x - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))


def record(obj, batch=False):
    v = ctypes.c_uint64()
    fn = nat.load().crsolve_batch_debug_bounds if batch else nat.load().crsolve_debug_bounds
    nat.check(fn(obj.handle, ctypes.byref(v), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
              "debug_bounds")
    return int(v.value)


def check_plan(plan, what):
    r = record(plan)
    if r != NONE:
        raise AssertionError(f"{what}: out-of-range access, level {r >> 56}, array {(r >> 48) & 0xFF}, "
                             f"index {r & 0xFFFFFFFFFFFF}")


def dev(*a):
    return [None if v is None else torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in a]


def main():
    assert nat.lib_path().endswith("libcrsolve_debug.so"), nat.lib_path()
    n = 0
    # plain FP64: sizes spanning tiles and ragged tails, every block-size class
    for N, m, k in [(1, 4, 1), (2, 3, 2), (3, 1, 1), (5, 8, 4), (17, 16, 3), (64, 4, 1), (129, 8, 5),
                    (1000, 4, 2), (33, 20, 17), (11, 32, 40), (9, 64, 33), (257, 12, 1)]:
        A, B, y = synthetic.gen_system(N, m, k, seed=N * m + k)
        dA, dB, dy = dev(A, B if N > 1 else None, y)
        plan = crs.Plan(N, m, k)
        crs.crsolve_factor(plan, dA, dB)
        x = crs.crsolve_solve(plan, dy).cpu().numpy()
        xo, io = oracle.cr_solve(A, B, y)
        assert crs.crsolve_info_get(plan) == io and rel(x, xo) <= TOL, (N, m, k)
        check_plan(plan, f"plain N={N} m={m} k={k}")
        n += 1
    # breakdown (NaN fill of x)
    A, B, y = synthetic.gen_system(64, 4, 2, seed=1)
    A = synthetic.make_indefinite(A, amount=1e3)
    dA, dB, dy = dev(A, B, y)
    plan = crs.Plan(64, 4, 2)
    crs.crsolve_factor(plan, dA, dB)
    x = crs.crsolve_solve(plan, dy)
    assert crs.crsolve_info_get(plan) == oracle.cr_solve(A, B, y)[1] and torch.isnan(x).all()
    check_plan(plan, "breakdown")
    n += 1
    # keep-levels plans: forward, scratch released, backward re-factors the coarse levels
    A, B, y = synthetic.gen_system(300, 8, 3, seed=5)
    c = synthetic.gen_cotangent(300, 8, 3, seed=5)
    dA, dB, dy, dc = dev(A, B, y, c)
    xo, _ = oracle.cr_solve(A, B, y)
    gyo, gAo, gBo, _ = oracle.cr_backward(A, B, xo, c)
    for keep in (0, 1, 3):
        plan = crs.Plan(300, 8, 3, keep_levels=keep)
        crs.crsolve_factor(plan, dA, dB)
        x = crs.crsolve_solve(plan, dy)
        plan.release_scratch()
        gy, gA, gB = crs.crsolve_backward(plan, x, dc)
        assert rel(x.cpu().numpy(), xo) <= TOL and rel(gy.cpu().numpy(), gyo) <= TOL
        assert rel(gA.cpu().numpy(), gAo) <= TOL and rel(gB.cpu().numpy(), gBo) <= TOL
        check_plan(plan, f"keep_levels {keep}")
        n += 1
    # host buffers (level 0-3 wavefront)
    A, B, y = synthetic.gen_system(2000, 8, 4, seed=6)
    plan = crs.Plan(2000, 8, 4, flags=nat.CRSOLVE_PLAN_HOST_STAGING)
    tx = torch.empty(2000, 8, 4, dtype=torch.complex128).pin_memory()
    crs.crsolve_solve_host(plan, *(torch.from_numpy(a).pin_memory() for a in (A, B, y)), tx)
    assert rel(tx.numpy(), oracle.cr_solve(A, B, y)[0]) <= TOL
    check_plan(plan, "host buffers")
    n += 1
    # mixed precision: CUDA-core and tensor-core classes (FP32 levels, split residuals)
    for N, m, k in [(300, 8, 4), (129, 64, 32), (77, 40, 3), (61, 57, 20), (65, 64, 40)]:
        A, B, y = synthetic.gen_system(N, m, k, seed=N + m)
        dA, dB, dy = dev(A, B, y)
        plan = crs.Plan(N, m, k, precision=nat.CRSOLVE_MIXED)
        crs.crsolve_factor(plan, dA, dB)
        x = crs.crsolve_solve(plan, dy).cpu().numpy()
        assert rel(x, oracle.cr_solve(A, B, y)[0]) <= 1e-10, (N, m, k)
        check_plan(plan, f"mixed N={N} m={m} k={k}")
        n += 1
    # Algorithm 1
    for N, m, k in [(1, 4, 1), (8, 4, 2), (64, 8, 3)]:
        A, B, y = synthetic.gen_system(N, m, k, seed=N + 3)
        dA, dB, dy = dev(A, B if N > 1 else None, y)
        plan = crs.Plan(N, m, k, flags=nat.CRSOLVE_PLAN_ALG1)
        crs.crsolve_factor(plan, dA, dB)
        x = crs.crsolve_solve(plan, dy).cpu().numpy()
        assert rel(x, oracle.alg1_solve(A, B, y)[0]) <= TOL, (N, m, k)
        check_plan(plan, f"alg1 N={N}")
        n += 1
    # batched: uneven N, m, k in one launch
    rng = np.random.default_rng(2)
    Ns = rng.integers(1, 200, 16)
    Ns[:3] = [1, 2, 129]
    ms = rng.choice([1, 3, 4, 8, 12, 16, 32], 16)
    ks = rng.integers(1, 17, 16)
    syss = [synthetic.gen_system(int(a), int(b), int(c), 90 + i) for i, (a, b, c) in enumerate(zip(Ns, ms, ks))]
    bt = crs.Batch(Ns, ms, ks)
    A, B, y = bt.pack(syss)
    x = crs.crsolve_batch_solve(bt, A, B, y)
    for i, s in enumerate(syss):
        assert rel(bt.system_view(i, A, B, x)[2].cpu().numpy(), oracle.cr_solve(*s)[0]) <= TOL, i
    r = record(bt, batch=True)
    assert r == NONE, f"batched: out-of-range access record {r:#x}"
    n += 1
    # the tensor-core residual on its own
    A, B, y = synthetic.gen_system(200, 64, 32, seed=8)
    xr = synthetic.gen_system(200, 64, 32, seed=9)[2]
    dA, dB, dx, dy = dev(A, B, xr, y)
    r1 = crs.crsolve_residual(dA, dB, dx, dy, method="split")
    r2 = crs.crsolve_residual(dA, dB, dx, dy, method="fp64")
    assert float((r1 - r2).abs().max()) <= 1e-12 * float(r2.abs().max())
    n += 1
    torch.cuda.synchronize()
    print(f"{n} cases ok")


if __name__ == "__main__":
    main()
