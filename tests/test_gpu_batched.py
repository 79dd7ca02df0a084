"""GPU parity of the batched form (one persistent launch over many systems of
uneven N, m, k) against the oracle, per system, and against the plain
single-system path (bit-identical: the same per-block arithmetic)."""
import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_1807_00370_gb300 as crs
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _systems(n, seed, n_lo=1, n_hi=300, ms=(1, 2, 3, 4, 5, 7, 8, 12, 16, 20, 32), k_hi=17):
    rng = np.random.default_rng(seed)
    Ns = rng.integers(n_lo, n_hi + 1, size=n)
    Ns[:6] = [1, 2, 3, 5, 64, 127][:min(6, n)]
    mm = rng.choice(np.asarray(ms), size=n)
    kk = rng.integers(1, k_hi + 1, size=n)
    syss = [synthetic.gen_system(int(N), int(m), int(k), seed * 1000 + i) for i, (N, m, k) in enumerate(zip(Ns, mm, kk))]
    return Ns, mm, kk, syss


def _plain(A, B, y):
    N, m, k = y.shape
    plan = crs.Plan(N, m, k)
    crs.crsolve_factor(plan, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda() if N > 1 else None)
    return crs.crsolve_solve(plan, torch.from_numpy(y).cuda()).cpu().numpy(), crs.crsolve_info_get(plan)


def test_offsets_match_the_generator_layout(cuda_ok):
    Ns, mm, kk, _ = _systems(10, 1)
    b = crs.Batch(Ns, mm, kk)
    oa, ob, oy, tot = synthetic.batch_offsets(Ns, mm, kk)
    assert np.array_equal(b.offA, oa) and np.array_equal(b.offB, ob) and np.array_equal(b.offY, oy)
    assert (b.nA, b.nB, b.nY) == tot


def test_uneven_batch_matches_oracle_and_plain_path(cuda_ok):
    Ns, mm, kk, syss = _systems(48, 2)
    b = crs.Batch(Ns, mm, kk)
    A, B, y = b.pack(syss)
    x = crs.crsolve_batch_solve(b, A, B, y)
    infos = crs.crsolve_batch_info(b)
    for i, (a, bb, yy) in enumerate(syss):
        xi = b.system_view(i, A, B, x)[2].cpu().numpy()
        xo, io = oracle.cr_solve(a, bb, yy)
        assert infos[i] == io and io["status"] == 0, i
        assert rel_err(xi, xo) <= TOL, i
        xp, _ = _plain(a, bb, yy)
        assert np.array_equal(xi, xp), f"system {i} (N={Ns[i]}, m={mm[i]}, k={kk[i]}) differs from the plain path"


def test_breakdown_flags_per_system(cuda_ok):
    Ns, mm, kk, syss = _systems(24, 3, n_lo=4, n_hi=200, ms=(2, 4, 8))
    bad = {1, 5, 11, 17}
    for i in bad:
        a, bb, yy = syss[i]
        a = a.copy()
        a[len(a) // 3] -= 50.0 * np.eye(a.shape[1])
        syss[i] = (a, bb, yy)
    b = crs.Batch(Ns, mm, kk)
    A, B, y = b.pack(syss)
    x = crs.crsolve_batch_solve(b, A, B, y)
    infos = crs.crsolve_batch_info(b)
    for i, (a, bb, yy) in enumerate(syss):
        xo, io = oracle.cr_solve(a, bb, yy)
        assert infos[i] == io, (i, infos[i], io)
        xi = b.system_view(i, A, B, x)[2].cpu().numpy()
        if i in bad:
            assert io["status"] == 1 and np.isnan(xi).all()
        else:
            assert rel_err(xi, xo) <= TOL


def test_graph_replay_equals_direct_launch(cuda_ok):
    Ns, mm, kk, syss = _systems(30, 4)
    b = crs.Batch(Ns, mm, kk)
    A, B, y = b.pack(syss)
    x1 = crs.crsolve_batch_solve(b, A, B, y)
    x2 = torch.empty_like(y)
    for _ in range(3):
        x2.zero_()
        crs.crsolve_batch_graph_launch(b, A, B, y, x2)
        torch.cuda.synchronize()
        assert torch.equal(x1, x2)


def test_fewer_slots_than_systems(cuda_ok):
    """A small workspace cap leaves two slots: every slot is reused many times."""
    Ns, mm, kk, syss = _systems(20, 5, n_hi=100)
    b0 = crs.Batch(Ns, mm, kk)
    per_slot = (b0.workspace_bytes - 65536) // max(b0.nslots, 1)
    b = crs.Batch(Ns, mm, kk, max_workspace_bytes=2 * per_slot + 65536)
    assert b.nslots <= 2
    A, B, y = b.pack(syss)
    x = crs.crsolve_batch_solve(b, A, B, y)
    for i, (a, bb, yy) in enumerate(syss):
        assert rel_err(b.system_view(i, A, B, x)[2], oracle.cr_solve(a, bb, yy)[0]) <= TOL


@pytest.mark.slow
def test_full_size_uneven_batch_sampled_against_oracle(cuda_ok):
    """4096 systems, N ~ U[16, 4096], m in {4, 8, 16, 32}, k ~ U[1, 16]: eight
    sampled systems against the oracle, every system by its residual."""
    Ns, mm, kk = synthetic.gen_batch_shapes(4096, seed=3003)
    A, B, y = synthetic.gen_batch_device(Ns, mm, kk, seed=3003)
    b = crs.Batch(Ns, mm, kk)
    x = crs.crsolve_batch_graph_launch(b, A, B, y, torch.empty_like(y))
    infos = crs.crsolve_batch_info(b)
    assert all(r["status"] == 0 for r in infos)
    rng = np.random.default_rng(0)
    big = int(np.argmax(Ns * mm.astype(np.int64) ** 3))
    for i in [big] + list(rng.choice(len(Ns), 7, replace=False)):
        a, bb, yy = (t.cpu().numpy() for t in b.system_view(i, A, B, y))
        xi = b.system_view(i, A, B, x)[2].cpu().numpy()
        assert rel_err(xi, oracle.cr_solve(a, bb, yy)[0]) <= TOL, i
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
    assert worst <= 1e-14
