"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # the library must load: a missing build is a failure, not a skip
    from paper_1802_07210_gb300 import _lib
    _lib.lib()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def grid_as_i32(g):
    return np.ascontiguousarray(g).view(np.int32)
