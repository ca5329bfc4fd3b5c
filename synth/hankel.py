"""Seeded block-Hankel test matrices built from Markov parameters h_k = C A^(k-1) B.

A is real, normal, with eigenvalues drawn uniformly (by area) in the disk of a
given radius, as conjugate pairs rho*exp(+-i*theta): A = V D V^T with D
block-diagonal of 2x2 rotation-scalings and V Haar orthogonal.  B and C are
standard Gaussian.  This is input construction only.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Tuple

import numpy as np

from .tucker import haar


@dataclass(frozen=True)
class HankelSpec:
    """A synthetic block-Hankel workload.

    order: state dimension of A (even: eigenvalues come in conjugate pairs)
    m, n:  block sizes (C is m x order, B is order x n); each block H_k is m x n
    s:     block rows = block columns; blocks k = 1..2s-1
    radius: eigenvalues of A lie in the disk of this radius
    r, ell_r, ell_l: target rank and the two sketch sizes
    """

    name: str
    order: int
    m: int
    n: int
    s: int
    radius: float
    data_seed: int
    r: int
    ell_r: int
    ell_l: int
    omega_seed: int = 0

    @property
    def nblocks(self) -> int:
        return 2 * self.s - 1

    @property
    def shape(self) -> Tuple[int, int]:
        return self.m * self.s, self.n * self.s


def hankel_config_spec(name: str = "c4") -> HankelSpec:
    """The 1024 x 1024 block Hankel of the build (128 x 128 blocks of 8 x 8)."""
    if name == "c4":
        return HankelSpec("c4", order=40, m=8, n=8, s=128, radius=0.95,
                          data_seed=1004, r=40, ell_r=50, ell_l=75)
    raise KeyError(name)


def system_matrices(spec: HankelSpec):
    """Draw (A, B, C) and the eigenvalues of A."""
    if spec.order % 2:
        raise ValueError("order must be even")
    rng = np.random.default_rng(spec.data_seed)
    npairs = spec.order // 2
    rho = spec.radius * np.sqrt(rng.random(npairs))
    theta = np.pi * rng.random(npairs)
    dmat = np.zeros((spec.order, spec.order))
    for p in range(npairs):
        c, s = rho[p] * np.cos(theta[p]), rho[p] * np.sin(theta[p])
        dmat[2 * p:2 * p + 2, 2 * p:2 * p + 2] = [[c, s], [-s, c]]
    v = haar(spec.order, spec.order, rng)
    a = v @ dmat @ v.T
    b = rng.standard_normal((spec.order, spec.n))
    cmat = rng.standard_normal((spec.m, spec.order))
    eig = np.concatenate([rho * np.exp(1j * theta), rho * np.exp(-1j * theta)])
    return a, b, cmat, eig


def markov_parameters(spec: HankelSpec) -> np.ndarray:
    """Blocks H_k = C A^(k-1) B, k = 1..2s-1, as a Fortran array (m, n, 2s-1).

    Block k (1-based) is ``blocks[:, :, k-1]``; each block is column-major.
    """
    a, b, cmat, _ = system_matrices(spec)
    out = np.zeros((spec.m, spec.n, spec.nblocks), order="F")
    akb = b.copy()  # A^(k-1) B
    for k in range(spec.nblocks):
        out[:, :, k] = cmat @ akb
        akb = a @ akb
    return out


def symmetric_markov_parameters(spec: HankelSpec) -> np.ndarray:
    """Blocks H_k = B^T A^(k-1) B of a symmetric system (A = A^T, C = B^T,
    m = n), k = 1..2s-1, Fortran array (m, m, 2s-1).  Block (i, j) of the
    block Hankel matrix is then (A^(i-1) B)^T (A^(j-1) B), so the matrix is
    K^T K with K = [B, A B, ..., A^(s-1) B]: symmetric positive semidefinite
    of rank <= order.  A = V diag(lambda) V^T with V Haar orthogonal and
    |lambda| uniform in [0.5, radius], random signs; B standard Gaussian."""
    if spec.m != spec.n:
        raise ValueError("a symmetric system needs m = n")
    rng = np.random.default_rng(spec.data_seed)
    lam = rng.uniform(0.5, spec.radius, spec.order) * rng.choice([-1.0, 1.0], spec.order)
    v = haar(spec.order, spec.order, rng)
    a = (v * lam) @ v.T
    b = rng.standard_normal((spec.order, spec.m))
    out = np.zeros((spec.m, spec.m, spec.nblocks), order="F")
    akb = b.copy()
    for k in range(spec.nblocks):
        out[:, :, k] = b.T @ akb
        akb = a @ akb
    return out


def two_level_markov_parameters(order: int, m: int, n: int, s1: int, s2: int, seed: int,
                                radius: float = 0.9) -> np.ndarray:
    """Blocks H_{k1,k2} = C diag(lambda^k1 mu^k2) B (k1 < 2 s1 - 1,
    k2 < 2 s2 - 1, 0-based) of a two-dimensional exponential sum, shape
    (m, n, 2 s1 - 1, 2 s2 - 1): the two-level block Hankel matrix they form
    is sum_r (u_r kron c_r)(v_r kron b_r)^T with Vandermonde-like u_r, v_r, so
    its rank is at most `order`.  lambda, mu uniform in [-radius, radius];
    B, C standard Gaussian.  Input construction only."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(-radius, radius, order)
    mu = rng.uniform(-radius, radius, order)
    b = rng.standard_normal((order, n))
    c = rng.standard_normal((m, order))
    out = np.zeros((m, n, 2 * s1 - 1, 2 * s2 - 1), order="F")
    for k1 in range(2 * s1 - 1):
        for k2 in range(2 * s2 - 1):
            out[:, :, k1, k2] = (c * (lam ** k1 * mu ** k2)) @ b
    return out
