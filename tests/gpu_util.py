"""Helpers for the GPU parity tests: layout conversion and comparisons.

Matrices cross the boundary column-major: a numpy (rows x cols) matrix A is
uploaded as torch.from_numpy(A.T) (shape (cols, rows), C-contiguous), which
has exactly A's column-major bytes.  Tensors use synth's layout helpers.
"""

import numpy as np
import pytest


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch


def dev():
    import torch
    return torch.device("cuda:0")


def mat_to_dev(a: np.ndarray, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a).T))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev())


def mat_from_dev(t, rows: int, cols: int) -> np.ndarray:
    import torch
    return t.detach().to(torch.float64).cpu().numpy().reshape(cols, rows).T.copy()


def empty_mat(rows: int, cols: int, dtype):
    import torch
    return torch.empty((cols, rows), dtype=dtype, device=dev())


def tensor_to_dev(x: np.ndarray, dtype):
    import torch
    from synth import to_torch_layout
    return to_torch_layout(np.asfortranarray(x)).to(dtype).to(dev())


def tensor_from_dev(t, dims) -> np.ndarray:
    import torch
    return np.asfortranarray(t.detach().to(torch.float64).cpu().numpy().reshape(dims[::-1]).T)


def rel(a, b) -> float:
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0))
