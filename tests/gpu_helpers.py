"""Shared helpers for the GPU parity tests (host <-> device marshalling)."""
import numpy as np
import pytest
import torch

from paper_2605_13209_b300 import gpchol


def require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def dev(a, dtype=torch.float64):
    """numpy (n,) or (n, m) -> column-major CUDA tensor."""
    a = np.asarray(a)
    if a.ndim == 1:
        a = a[:, None]
    t = gpchol.colmajor(a.shape[0], a.shape[1], dtype=dtype)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return t


def host(t):
    return np.asfortranarray(t.detach().cpu().double().numpy())


@pytest.fixture(scope="session")
def ctx():
    require_gpu()
    c = gpchol.Context(0)
    yield c
    c.close()
