"""The bounded device-side wait of the tensor-core kernels (mbar_wait): a wait
on an mbarrier that nothing arrives at gives up after its poll limit and the
host gets CRSOLVE_ETIMEOUT; the context stays usable (a solve afterwards
matches the oracle).  No MMA and no tensor memory are involved, so nothing is
released while work is in flight."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synthetic
import paper_1807_00370_gb300 as crs
from paper_1807_00370_gb300 import _native as nat

pytestmark = pytest.mark.gpu


def test_wait_on_a_barrier_nothing_arrives_at_times_out(cuda_ok):
    ws = torch.empty(4, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for polls in (1, 100, 10000):
        rc = nat.load().crsolve_check_bounded_wait(polls, ctypes.c_void_p(ws.data_ptr()), stream)
        assert rc == nat.CRSOLVE_ETIMEOUT, rc
    A, B, y = synthetic.gen_system(65, 64, 8, seed=3)
    x = crs.solve(*(torch.from_numpy(a).cuda() for a in (A, B, y))).cpu().numpy()
    xo, _ = oracle.cr_solve(A, B, y)
    assert np.linalg.norm(x - xo) <= 1e-12 * np.linalg.norm(xo)
