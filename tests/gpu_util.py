"""Helpers shared by the GPU tests (device transfer, builds); no arithmetic of the method."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as entry

    entry.build()
    return torch.device("cuda:0")


def to_dev(a, d):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=d)


def panel(n, k, d):
    """An n x k column-major float64 panel (columns contiguous)."""
    return torch.zeros((k, n), dtype=torch.float64, device=d).t()


def relerr(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
