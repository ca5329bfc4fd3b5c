"""Kronecker / Khatri-Rao products, unfoldings, TTM and MTTKRP by definition (Sec. 2.1).

Conventions (Sec. 2.1 and Def. of KRP, Sec. 2.5), indices 0-based:
  * a tensor X of dims (n_1..n_d) is a numpy array of that shape;
  * the mode-n unfolding X_(n) is n_n x prod_{j!=n} n_j whose column index is
    sum_{j != n} i_j * J_j with J_j = prod_{m < j, m != n} n_m (first remaining
    mode fastest), so that the TTM identity
    Y_(n) = A_n X_(n) (A_d kron ... kron A_{n+1} kron A_{n-1} kron ... kron A_1)
    of Sec. 2.1 holds;
  * (A kron B) is the block matrix [a_ij B]; (A kr B) has column k equal to
    a_k kron b_k, so the row index of A kr B is (i_A, i_B) with i_A slowest.
"""

from __future__ import annotations

from functools import reduce
from typing import Sequence

import numpy as np


def kron(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Kronecker product as the block matrix [a_ij * B] (Sec. 2.1)."""
    ma, na = a.shape
    mb, nb = b.shape
    out = np.zeros((ma * mb, na * nb))
    for i in range(ma):
        for j in range(na):
            out[i * mb:(i + 1) * mb, j * nb:(j + 1) * nb] = a[i, j] * b
    return out


def khatri_rao(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Column-wise Kronecker product: column k is a[:,k] kron b[:,k] (Sec. 2.1)."""
    if a.shape[1] != b.shape[1]:
        raise ValueError("Khatri-Rao factors need the same number of columns")
    ell = a.shape[1]
    out = np.empty((a.shape[0] * b.shape[0], ell))
    for k in range(ell):
        out[:, k] = np.kron(a[:, k], b[:, k])
    return out


def khatri_rao_list(mats: Sequence[np.ndarray]) -> np.ndarray:
    """A_1 kr A_2 kr ... kr A_m (left to right; A_1's row index slowest)."""
    return reduce(khatri_rao, mats)


def krp_except(omegas: Sequence[np.ndarray], n: int) -> np.ndarray:
    """K_n = Omega_d kr ... kr Omega_{n+1} kr Omega_{n-1} kr ... kr Omega_1.

    The sketching matrix of the mode-n MTTKRP in Alg. 7 and Alg. 8 (0-based n).
    Its row index is the column index of X_(n): mode 1 fastest.
    """
    order = [omegas[j] for j in range(len(omegas) - 1, -1, -1) if j != n]
    return khatri_rao_list(order)


def unfold(x: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding X_(n) with the column order of Sec. 2.1."""
    return np.reshape(np.moveaxis(x, n, 0), (x.shape[n], -1), order="F")


def fold(m: np.ndarray, n: int, dims: Sequence[int]) -> np.ndarray:
    """Inverse of unfold: the tensor of dims ``dims`` whose X_(n) is ``m``."""
    dims = list(dims)
    moved = [dims[n]] + dims[:n] + dims[n + 1:]
    return np.moveaxis(np.reshape(m, moved, order="F"), 0, n)


def ttm(x: np.ndarray, a: np.ndarray, n: int) -> np.ndarray:
    """Y = X x_n A, defined by Y_(n) = A X_(n) (Sec. 2.1)."""
    dims = list(x.shape)
    dims[n] = a.shape[0]
    return fold(a @ unfold(x, n), n, dims)


def multi_ttm(x: np.ndarray, mats: Sequence[np.ndarray]) -> np.ndarray:
    """X x_1 A_1 x_2 A_2 ... x_d A_d by successive unfold-multiply-fold steps."""
    y = x
    for n, a in enumerate(mats):
        if a is not None:
            y = ttm(y, a, n)
    return y


def mttkrp(x: np.ndarray, omegas: Sequence[np.ndarray], n: int) -> np.ndarray:
    """Y_n = X_(n) K_n with the Khatri-Rao product formed explicitly (Alg. 7)."""
    return unfold(x, n) @ krp_except(omegas, n)


def frob(x: np.ndarray) -> float:
    """Frobenius norm sqrt(sum x^2) (Sec. 2.1)."""
    return float(np.sqrt(np.sum(np.square(x, dtype=np.float64))))
