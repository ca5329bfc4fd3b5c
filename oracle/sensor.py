"""Sensor placement from Tucker factors (Sec. 6), FP64 on the host.

Test-infrastructure only: the CUDA library never imports this module.

Training phase (Sec. 6): for each spatial mode i, with Q_i (N_i x l_i,
orthonormal columns) from a Tucker approximation of the snapshot tensor,
a column-pivoted QR of Q_i^T picks l_i columns of the identity, P_i; the
interpolation factor is A_i = Q_i (P_i^T Q_i)^{-1}.  Test phase: a new field T
is measured at the grid I_1 x ... x I_d only, T_hat = T(I_1, ..., I_d), and
T ~ T_hat x_1 A_1 ... x_d A_d.
"""

from __future__ import annotations

from typing import Sequence

import numpy as np

from .tucker import reconstruct


def pivoted_qr_select(q: np.ndarray) -> np.ndarray:
    """The first l pivots of the column-pivoted Householder QR of Q^T (l x N).

    Step k (k = 0..l-1): among columns k..N-1 of the working matrix W = Q^T
    (as reduced by steps 0..k-1), take the one whose part in rows k..l-1 has
    the largest 2-norm (ties: the lowest position), swap it into position k,
    and apply the Householder reflector that maps W[k:, k] onto
    alpha e_1 (alpha = -sign(W[k, k]) ||W[k:, k]||, sign(0) = +1) to columns
    k..N-1.  Returns the original column indices of positions 0..l-1, in the
    order they were picked.
    """
    w = np.array(q.T, dtype=np.float64, copy=True)
    ell, n = w.shape
    perm = np.arange(n)
    for k in range(ell):
        norms = np.sum(w[k:, k:] * w[k:, k:], axis=0)
        j = k + int(np.argmax(norms))
        if j != k:
            w[:, [k, j]] = w[:, [j, k]]
            perm[[k, j]] = perm[[j, k]]
        x = w[k:, k]
        nx = np.sqrt(np.dot(x, x))
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        vv = np.dot(v, v)
        if vv > 0.0:
            w[k:, k:] -= np.outer(v, (2.0 / vv) * (v @ w[k:, k:]))
    return perm[:ell].copy()


def interpolation_factor(q: np.ndarray, idx: Sequence[int]) -> np.ndarray:
    """A = Q (P^T Q)^{-1}, with P^T Q = Q[idx, :] (a linear solve)."""
    b = q[np.asarray(idx), :]
    return np.linalg.solve(b.T, q.T).T


def sensor_reconstruct(t_hat: np.ndarray, factors: Sequence[np.ndarray]) -> np.ndarray:
    """T_hat x_1 A_1 ... x_d A_d."""
    return reconstruct(t_hat, factors)


def pivot_margins(q: np.ndarray) -> np.ndarray:
    """For each step of pivoted_qr_select, (largest - second largest) / largest
    of the candidate norms: a decision with a margin near the rounding level
    may flip under another summation order (used by the tests to keep their
    inputs away from such ties)."""
    w = np.array(q.T, dtype=np.float64, copy=True)
    ell, n = w.shape
    out = []
    for k in range(ell):
        norms = np.sum(w[k:, k:] * w[k:, k:], axis=0)
        srt = np.sort(norms)[::-1]
        out.append((srt[0] - srt[1]) / srt[0] if srt.size > 1 and srt[0] > 0 else 1.0)
        j = k + int(np.argmax(norms))
        if j != k:
            w[:, [k, j]] = w[:, [j, k]]
        x = w[k:, k]
        nx = np.sqrt(np.dot(x, x))
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        vv = np.dot(v, v)
        if vv > 0.0:
            w[k:, k:] -= np.outer(v, (2.0 / vv) * (v @ w[k:, k:]))
    return np.array(out)
