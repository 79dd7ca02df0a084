"""Shared helpers of the GPU parity tests (inputs from synthetic, references from oracle)."""
import numpy as np
import torch


def to_dev(*arrs):
    return [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def rel_err(x, ref):
    x = x.cpu().numpy() if isinstance(x, torch.Tensor) else x
    return float(np.linalg.norm((x - ref).ravel()) / np.linalg.norm(ref.ravel()))
