"""The Cauchy tensor of the paper's Tucker experiments (Sec. 5.3):

    x[i_1, ..., i_d] = 1 / (i_1^alpha + ... + i_d^alpha)^(1/alpha),  1 <= i_j <= n,

a deterministic input (no random draws).  Smaller alpha gives sharper decay of
the mode-wise singular values.  Input construction only.
"""

from __future__ import annotations

import numpy as np


def cauchy_tensor(n: int, d: int = 4, alpha: float = 2.0) -> np.ndarray:
    """FP64 host array of shape (n,) * d in Fortran order (the tensor is
    symmetric in its indices, so every layout holds the same values)."""
    v = np.arange(1, n + 1, dtype=np.float64) ** alpha
    s = np.zeros((n,) * d)
    for j in range(d):
        shape = [1] * d
        shape[j] = n
        s = s + v.reshape(shape)
    return np.asfortranarray(s ** (-1.0 / alpha))


def cauchy_tensor_device(n: int, d: int = 4, alpha: float = 2.0, device="cuda", dtype=None,
                         slabs_per_chunk: int = 8):
    """The same values as a contiguous torch tensor of shape (n,) * d on the
    device, computed in FP64 a few slabs of the last index at a time and
    stored as ``dtype`` (FP32 by default)."""
    import torch
    dtype = dtype or torch.float32
    v = torch.arange(1, n + 1, dtype=torch.float64, device=device) ** alpha
    inner = torch.zeros((n,) * (d - 1), dtype=torch.float64, device=device)
    for j in range(d - 1):
        shape = [1] * (d - 1)
        shape[j] = n
        inner = inner + v.reshape(shape)
    out = torch.empty((n,) * d, dtype=dtype, device=device)
    for t0 in range(0, n, slabs_per_chunk):
        t1 = min(n, t0 + slabs_per_chunk)
        s = inner.unsqueeze(0) + v[t0:t1].reshape((t1 - t0,) + (1,) * (d - 1))
        out[t0:t1] = (s ** (-1.0 / alpha)).to(dtype)
    return out
