"""Shared helpers of the GPU tests (import only from tests)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_dev(p):
    dev = torch.device("cuda:0")
    return (torch.from_numpy(p.d).to(dev), torch.from_numpy(p.Ndiag).to(dev),
            torch.from_numpy(p.mask).to(dev), torch.from_numpy(p.Pk).to(dev))


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
