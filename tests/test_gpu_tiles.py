"""Every tile shape that the benchmark or the autotuner can time is checked
against the oracle.

- The plain path's process-wide tile table (crsolve_tile_set): each parameter
  of every block-size class varied over its swept range, plus random
  combinations, through the full factor + solve parity check; the defaults
  are restored afterwards.
- The batched form's autotuner: every (nb_factor, nb_solve, kc) the tuner
  times for a class, and the tile it picks, on a batch of that class.
- The full 4096-system batch with tiles="auto", the configuration the
  benchmark times.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_1807_00370_gb300 as crs
from paper_1807_00370_gb300 import _native as nat
from paper_1807_00370_gb300 import autotune
from tests.gpu_helpers import rel_err, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-12
NB = (1, 2, 3, 4, 8, 16, 32, 64)
KC = (1, 4, 8, 16, 32)
THREADS = (64, 128, 192, 256)


def _solve(A, B, y):
    N, m, k = y.shape
    dA, dB, dy = to_dev(A, B, y)
    plan = crs.Plan(N, m, k)
    crs.crsolve_factor(plan, dA, dB)
    x = crs.crsolve_solve(plan, dy).cpu().numpy()
    return x, crs.crsolve_info_get(plan)


def _shapes(m):
    """Tile shapes of class m: one parameter at a time around the default, then
    random combinations (shapes that do not fit are rejected by the library)."""
    base = list(crs.crsolve_tile_get(m))   # (nb_factor, nb_solve, kc, threads, threads_solve)
    out = []
    for i, rng_vals in enumerate((NB, NB, KC, THREADS, THREADS)):
        for v in rng_vals:
            s = list(base)
            s[i] = v
            out.append(tuple(s))
    rng = np.random.default_rng(m)
    for _ in range(12):
        out.append((int(rng.choice(NB)), int(rng.choice(NB)), int(rng.choice(KC)), int(rng.choice(THREADS)),
                    int(rng.choice(THREADS))))
    return base, list(dict.fromkeys(out))


@pytest.mark.parametrize("m", [4, 8, 16, 32, 64])
def test_plain_tile_shapes_match_oracle(cuda_ok, m):
    N, k = (1000, 19) if m <= 16 else (203, 19)
    A, B, y = synthetic.gen_system(N, m, k, seed=11 * m)
    xo, io = oracle.cr_solve(A, B, y)
    base, shapes = _shapes(m)
    tried = 0
    try:
        for s in shapes:
            try:
                crs.crsolve_tile_set(m, *s)
            except nat.CrsolveError:
                continue                          # out of range or too large for shared memory
            x, info = _solve(A, B, y)
            assert info == io, s
            assert rel_err(x, xo) <= TOL, s
            tried += 1
    finally:
        crs.crsolve_tile_set(m, *base)
    assert list(crs.crsolve_tile_get(m)) == base
    assert tried >= 10, tried


def _class_batch(m, seed, n=12):
    rng = np.random.default_rng(seed)
    Ns = rng.integers(1, 400, size=n)
    Ns[:3] = [1, 2, 129]
    ms = np.full(n, m)
    ks = rng.integers(1, 17, size=n)
    syss = [synthetic.gen_system(int(N), m, int(k), seed * 100 + i) for i, (N, k) in enumerate(zip(Ns, ks))]
    return Ns, ms, ks, syss


@pytest.mark.parametrize("m", [4, 8, 16, 32])
def test_autotuner_candidates_and_choice_match_oracle(cuda_ok, m):
    """tune_class on a small sample: the tile it returns and every tile it
    timed give the oracle's answer on a batch of the class."""
    best, table = autotune.tune_class(m, m, 8, n_blocks=64)
    cands = {tuple(best)}
    for nbf in table["factor"]:
        cands.add((int(nbf), 1, 8))
    for key in table["solve"]:
        nbs, kc = (int(v) for v in key.split(","))
        cands.add((int(best[0]), nbs, kc))
    Ns, ms, ks, syss = _class_batch(m, seed=40 + m)
    ref = [oracle.cr_solve(*s) for s in syss]
    for tile in sorted(cands):
        b = crs.Batch(Ns, ms, ks, tiles={m: tile})
        A, B, y = b.pack(syss)
        x = crs.crsolve_batch_solve(b, A, B, y)
        infos = crs.crsolve_batch_info(b)
        for i, (xo, io) in enumerate(ref):
            assert infos[i] == io, (tile, i)
            assert rel_err(b.system_view(i, A, B, x)[2].cpu().numpy(), xo) <= TOL, (tile, i)
        b.close()


@pytest.mark.slow
def test_full_batch_with_autotuned_tiles_as_benchmarked(cuda_ok):
    """The benchmark's batched workload exactly as it is timed: 4096 systems
    (seed 3003), Batch(..., tiles="auto"), CUDA graph replay; sampled systems
    against the oracle and every system by its residual."""
    Ns, mm, kk = synthetic.gen_batch_shapes(4096, seed=3003)
    A, B, y = synthetic.gen_batch_device(Ns, mm, kk, seed=3003)
    b = crs.Batch(Ns, mm, kk, tiles="auto")
    x = torch.empty_like(y)
    for _ in range(2):
        crs.crsolve_batch_graph_launch(b, A, B, y, x)
    infos = crs.crsolve_batch_info(b)
    assert all(r["status"] == 0 for r in infos)
    rng = np.random.default_rng(1)
    for cls in (4, 8, 16, 32):
        idx = np.flatnonzero(mm == cls)
        for i in rng.choice(idx, 2, replace=False):
            a, bb, yy = (t.cpu().numpy() for t in b.system_view(int(i), A, B, y))
            xi = b.system_view(int(i), A, B, x)[2].cpu().numpy()
            assert rel_err(xi, oracle.cr_solve(a, bb, yy)[0]) <= TOL, (cls, i, b.tiles)
    worst = 0.0
    for i in range(len(Ns)):
        a, bb, xi = b.system_view(i, A, B, x)
        yi = b.system_view(i, A, B, y)[2]
        Ah = torch.tril(a, -1)
        Ah = Ah + Ah.conj().transpose(1, 2) + torch.diag_embed(torch.diagonal(a, dim1=1, dim2=2).real.to(a.dtype))
        r = yi - torch.bmm(Ah, xi)
        if len(bb):
            r[1:] -= torch.bmm(bb, xi[:-1])
            r[:-1] -= torch.bmm(bb.conj().transpose(1, 2), xi[1:])
        nA = (Ah.abs().sum(2).max() + 2 * (bb.abs().sum(2).max() if len(bb) else 0)).item()
        worst = max(worst, (r.abs().amax() / (nA * xi.abs().amax())).item())
    assert worst <= 1e-14, (worst, b.tiles)


@pytest.mark.parametrize("m,k,prec", [(8, 4, 0), (16, 8, 0), (64, 32, 1)])
def test_plan_autotuner_choice_matches_oracle(cuda_ok, m, k, prec):
    """plan_tiles tunes the plan kernels' tile table for (class, k, precision)
    on a sample system, writes the choice into the table, and that table
    solves a fresh system to the oracle's answer (FP64 at 1e-12, mixed at
    the stated 1e-10); the table is restored afterwards."""
    get = crs.crsolve_tile_get_mixed if prec else crs.crsolve_tile_get
    put = crs.crsolve_tile_set_mixed if prec else crs.crsolve_tile_set
    before = get(m)
    try:
        shape = autotune.plan_tiles(m, k, prec, use_cache=False, apply=True)
        assert get(m) == shape
        N = 777 if m < 64 else 129
        A, B, y = synthetic.gen_system(N, m, k, seed=5 * m + k)
        dA, dB, dy = to_dev(A, B, y)
        plan = crs.Plan(N, m, k, precision=prec)
        crs.crsolve_factor(plan, dA, dB)
        x = crs.crsolve_solve(plan, dy).cpu().numpy()
        xo, io = oracle.cr_solve(A, B, y)
        assert crs.crsolve_info_get(plan) == io
        assert rel_err(x, xo) <= (1e-10 if prec else TOL), shape
    finally:
        put(m, *before)
    assert get(m) == before
