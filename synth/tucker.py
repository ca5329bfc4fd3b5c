"""Seeded Tucker-structured test tensors (core times orthonormal factors, plus noise).

The workloads follow the synthetic configurations of the build: a random core
G0 (optionally with geometric decay), Haar-distributed orthonormal factors U_i,
X0 = G0 x_1 U_1 ... x_d U_d, and additive Gaussian noise of a prescribed
relative Frobenius norm.  This is input construction only.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclass(frozen=True)
class TuckerSpec:
    """A synthetic Tucker workload.

    dims:   tensor sides (n_1, ..., n_d)
    core:   multilinear rank of the noise-free part (sides of G0)
    noise:  relative Frobenius norm of the additive noise (0 = none)
    decay:  None, or q so that G0[i_1..i_d] = N(0,1) * q**(i_1+...+i_d), 0-based
    data_seed: seed of the numpy stream that draws G0, U_i and the noise
    ranks:  target multilinear rank r_i of the approximation
    ell:    sketch sizes l_i = r_i + oversampling
    omega_seed: Philox seed of the sketching factors
    """

    name: str
    dims: Tuple[int, ...]
    core: Tuple[int, ...]
    noise: float
    decay: Optional[float]
    data_seed: int
    ranks: Tuple[int, ...]
    ell: Tuple[int, ...]
    omega_seed: int = 0

    @property
    def d(self) -> int:
        return len(self.dims)

    @property
    def numel(self) -> int:
        return int(np.prod(self.dims, dtype=np.int64))

    @property
    def oversample(self) -> int:
        return self.ell[0] - self.ranks[0]


def config_spec(name: str) -> TuckerSpec:
    """Named synthetic workloads (sizes and seeds of the build's configurations)."""
    if name == "c1":   # 64^3, exact rank 5 + 1e-6 noise, l = 10
        return TuckerSpec("c1", (64, 64, 64), (5, 5, 5), 1e-6, None, 1001,
                          (5, 5, 5), (10, 10, 10))
    if name == "c2":   # 1024^3, rank 32 + 1e-4 noise, l = 48
        return TuckerSpec("c2", (1024, 1024, 1024), (32, 32, 32), 1e-4, None,
                          1002, (32, 32, 32), (48, 48, 48))
    if name == "c3":   # 200^4, decaying 40^4 core, no noise, r = 20, l = 30
        return TuckerSpec("c3", (200, 200, 200, 200), (40, 40, 40, 40), 0.0,
                          0.8, 1003, (20, 20, 20, 20), (30, 30, 30, 30))
    raise KeyError(name)


def haar(n: int, r: int, rng: np.random.Generator) -> np.ndarray:
    """n x r matrix with orthonormal columns, Haar distributed.

    Orthonormalises an n x r standard Gaussian with numpy's LAPACK QR and folds
    the signs of diag(R) into the columns, which makes the result Haar.
    """
    g = rng.standard_normal((n, r))
    q, rr = np.linalg.qr(g)
    s = np.sign(np.diag(rr))
    s[s == 0] = 1.0
    return q * s[None, :]


def tucker_factors(spec: TuckerSpec) -> Tuple[np.ndarray, List[np.ndarray]]:
    """Draw the core G0 (Fortran order) and the orthonormal factors U_i."""
    rng = np.random.default_rng(spec.data_seed)
    g0 = rng.standard_normal(spec.core[::-1]).T  # Fortran-ordered view
    g0 = np.asfortranarray(g0)
    if spec.decay is not None:
        idx = np.zeros(spec.core, dtype=np.float64)
        for ax, r in enumerate(spec.core):
            shape = [1] * len(spec.core)
            shape[ax] = r
            idx = idx + np.arange(r, dtype=np.float64).reshape(shape)
        g0 = np.asfortranarray(g0 * spec.decay ** idx)
    us = [haar(n, r, rng) for n, r in zip(spec.dims, spec.core)]
    return g0, us


def _ttm_np(x: np.ndarray, u: np.ndarray, mode: int) -> np.ndarray:
    y = np.tensordot(u, x, axes=(1, mode))
    return np.moveaxis(y, 0, mode)


def expand_tucker(g0: np.ndarray, us: Sequence[np.ndarray]) -> np.ndarray:
    """X0 = G0 x_1 U_1 ... x_d U_d on the host, FP64, Fortran order."""
    x = g0
    for mode, u in enumerate(us):
        x = _ttm_np(x, u, mode)
    return np.asfortranarray(x)


def _noise_rng(spec: TuckerSpec) -> np.random.Generator:
    return np.random.default_rng([spec.data_seed, 7])


def tucker_tensor(spec: TuckerSpec):
    """Host FP64 tensor (Fortran order) plus its generating factors.

    Noise: E = eps * ||X0||_F * E0 / ||E0||_F with E0 i.i.d. N(0,1).
    Returns (X, G0, [U_i]).
    """
    g0, us = tucker_factors(spec)
    x0 = expand_tucker(g0, us)
    if spec.noise > 0:
        rng = _noise_rng(spec)
        e0 = np.asfortranarray(rng.standard_normal(spec.dims[::-1]).T)
        x0 = x0 + spec.noise * np.linalg.norm(x0) * e0 / np.linalg.norm(e0)
    return np.asfortranarray(x0), g0, us


def tucker_tensor_device(spec: TuckerSpec, device="cuda", chunk_elems=1 << 28):
    """Full-size tensor expanded on a CUDA device, FP64, torch layout (n_d..n_1).

    The small factors come from the same numpy stream as tucker_tensor(); the
    expansion runs as torch tensordots on the device and the noise is drawn from
    a seeded torch.Generator on that device (deterministic for a given device
    and torch build, not bit-identical to the host variant).
    Returns (X_t, G0, [U_i]).
    """
    import torch

    g0, us = tucker_factors(spec)
    d = spec.d
    xt = torch.from_numpy(np.ascontiguousarray(g0.T)).to(device)  # (r_d..r_1)
    for mode, u in enumerate(us):
        ut = torch.from_numpy(u).to(device)
        tdim = d - 1 - mode
        xt = torch.movedim(torch.tensordot(ut, xt, dims=([1], [tdim])), 0, tdim)
        xt = xt.contiguous()
    if spec.noise > 0:
        gen = torch.Generator(device=device)
        gen.manual_seed(spec.data_seed * 7919 + 7)
        flat = xt.view(-1)
        x_norm = torch.linalg.vector_norm(flat).item()
        # E0 is drawn chunk by chunk twice from the same generator state: once
        # for its norm, once to add it, so only one chunk is resident at a time.
        state = gen.get_state()
        e_sq = 0.0
        for start in range(0, flat.numel(), chunk_elems):
            stop = min(start + chunk_elems, flat.numel())
            e = torch.randn(stop - start, generator=gen, device=device,
                            dtype=torch.float64)
            e_sq += float(torch.dot(e, e).item())
        scale = spec.noise * x_norm / np.sqrt(e_sq)
        gen.set_state(state)
        for start in range(0, flat.numel(), chunk_elems):
            stop = min(start + chunk_elems, flat.numel())
            e = torch.randn(stop - start, generator=gen, device=device,
                            dtype=torch.float64)
            flat[start:stop].add_(e, alpha=scale)
    return xt, g0, us


def to_torch_layout(x: np.ndarray):
    """Fortran-ordered numpy (n_1..n_d) -> C-contiguous torch (n_d..n_1), no copy."""
    import torch

    return torch.from_numpy(np.ascontiguousarray(x.T))


def from_torch_layout(t) -> np.ndarray:
    """torch (n_d..n_1) -> Fortran-ordered numpy (n_1..n_d) on the host."""
    return np.asfortranarray(t.detach().cpu().numpy().T)
