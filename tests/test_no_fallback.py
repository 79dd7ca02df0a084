"""Host-side guarantees that need no GPU: without a CUDA device the solver
raises instead of computing anything on the CPU (there is no CPU fallback in
the package), and CRSolveFn rejects invalid keep_factors values before any
device work."""
import numpy as np
import pytest
import torch

import synthetic
import paper_1807_00370_gb300 as crs


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a CUDA device")
@pytest.mark.parametrize("where", ["host tensors", "plan"])
def test_no_cpu_fallback_without_a_gpu(where):
    A, B, y = (torch.from_numpy(a) for a in synthetic.gen_system(16, 4, 2, seed=1))
    with pytest.raises(RuntimeError):
        if where == "host tensors":
            crs.solve(A, B, y)
        else:
            crs.Plan(16, 4, 2)


@pytest.mark.parametrize("keep", [-1, -5])
def test_keep_factors_must_be_a_level_count(keep):
    A, B, y = (torch.from_numpy(a) for a in synthetic.gen_system(16, 4, 2, seed=2))
    with pytest.raises(ValueError):
        crs.CRSolveFn.apply(A, B, y, keep)


def test_keep_levels_needs_the_classic_method():
    A, B, y = (torch.from_numpy(a) for a in synthetic.gen_system(16, 4, 2, seed=3))
    with pytest.raises(ValueError):
        crs.CRSolveFn.apply(A, B, y, 2, "alg1")
