"""Helpers shared by the GPU tests (device tensors, library context)."""
import numpy as np
import pytest


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def ctx():
    from paper_2511_18207_gb300 import prohd

    return prohd.context()


def dev(x):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.fixture
def prune_always():
    """Row pruning at any contraction size (the default threshold, 4e9
    row-column pairs, would leave oracle-sized cases on the plain path)."""
    c = ctx()
    c.set_prune_min_pairs(0.0)
    yield c
    c.set_prune_min_pairs(4e9)
