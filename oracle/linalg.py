"""Dense FP64 kernels of the oracle: Householder thin QR, one-sided Jacobi SVD,
two-sided Jacobi eigen-decomposition, LS.

The thin QR Y = QR is the orthonormalisation step of the randomized range
finder (Alg. 1) and of every sketch in Alg. 6, 7 and 8.  It is written out as
Householder QR (no Cholesky/Gram route, so exactly rank-deficient sketches stay
well defined) with the sign convention diag(R) >= 0.
"""

from __future__ import annotations

import numpy as np


def householder_qr(y: np.ndarray):
    """Thin QR of an m x l matrix (m >= l): returns Q (m x l), R (l x l).

    Reflector j zeroes column j below the diagonal: x = A[j:, j],
    alpha = -sign(x_0) ||x||, v = x - alpha e_1, A[j:, j:] -= (2/v'v) v (v' A[j:, j:]).
    Q is accumulated by applying the reflectors in reverse order to [I; 0].
    Finally the signs are flipped so that diag(R) >= 0.
    """
    a = np.array(y, dtype=np.float64, copy=True)
    m, l = a.shape
    if m < l:
        raise ValueError("thin QR needs rows >= columns")
    vs = []
    taus = []
    for j in range(l):
        x = a[j:, j].copy()
        normx = np.sqrt(np.dot(x, x))
        if normx == 0.0:
            vs.append(np.zeros_like(x))
            taus.append(0.0)
            continue
        alpha = -normx if x[0] >= 0 else normx
        v = x.copy()
        v[0] -= alpha
        vtv = np.dot(v, v)
        tau = 2.0 / vtv if vtv > 0 else 0.0
        a[j:, j:] -= tau * np.outer(v, v @ a[j:, j:])
        vs.append(v)
        taus.append(tau)
    r = np.triu(a[:l, :l])
    q = np.zeros((m, l))
    q[:l, :l] = np.eye(l)
    for j in range(l - 1, -1, -1):
        v = vs[j]
        q[j:, :] -= taus[j] * np.outer(v, v @ q[j:, :])
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :], r * s[:, None]


def jacobi_svd(a: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Thin SVD by one-sided (Hestenes) Jacobi rotations on the columns.

    Rotates column pairs (p, q) of W = A (m x n, m >= n) until all pairs are
    orthogonal to ``tol`` relative; then sigma_k = ||w_k||, u_k = w_k / sigma_k
    and V accumulates the rotations.  Returns U (m x n), s (n, descending), Vt.
    For m < n it factors A^T and swaps the roles of U and V.
    """
    a = np.array(a, dtype=np.float64, copy=True)
    m, n = a.shape
    if m < n:
        u, s, vt = jacobi_svd(a.T, tol, max_sweeps)
        return vt.T, s, u.T
    w = a
    v = np.eye(n)
    for _ in range(max_sweeps):
        off = 0.0
        for p in range(n - 1):
            for q in range(p + 1, n):
                alpha = np.dot(w[:, p], w[:, p])
                beta = np.dot(w[:, q], w[:, q])
                gamma = np.dot(w[:, p], w[:, q])
                if alpha == 0.0 or beta == 0.0:
                    continue
                c_rel = abs(gamma) / np.sqrt(alpha * beta)
                off = max(off, c_rel)
                if c_rel <= tol:
                    continue
                zeta = (beta - alpha) / (2.0 * gamma)
                t = np.sign(zeta) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                if zeta == 0.0:
                    t = 1.0
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                wp = w[:, p].copy()
                w[:, p] = c * wp - s * w[:, q]
                w[:, q] = s * wp + c * w[:, q]
                vp = v[:, p].copy()
                v[:, p] = c * vp - s * v[:, q]
                v[:, q] = s * vp + c * v[:, q]
        if off <= tol:
            break
    sig = np.sqrt(np.sum(w * w, axis=0))
    order = np.argsort(-sig, kind="stable")
    sig = sig[order]
    w = w[:, order]
    v = v[:, order]
    u = np.zeros_like(w)
    for k in range(n):
        if sig[k] > 0:
            u[:, k] = w[:, k] / sig[k]
    return u, sig, v.T


def jacobi_eig(a: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Eigen-decomposition of a symmetric matrix by the cyclic two-sided
    (classical) Jacobi method.

    Each rotation J in the plane (p, q) is chosen so that (J^T A J)_pq = 0:
    theta = (a_qq - a_pp) / (2 a_pq), t = sign(theta) / (|theta| +
    sqrt(1 + theta^2)) (t = 1 when theta = 0), c = 1 / sqrt(1 + t^2), s = t c;
    columns p, q and then rows p, q of A are rotated, and V accumulates the
    columns.  Sweeps stop when the off-diagonal Frobenius norm is at most
    ``tol`` times that of A.  Returns the eigenvalues in descending order
    (negative ones included) and V with the eigenvectors as columns.
    """
    a = np.array(a, dtype=np.float64, copy=True)
    a = 0.5 * (a + a.T)
    n = a.shape[0]
    v = np.eye(n)
    scale = np.linalg.norm(a)
    for _ in range(max_sweeps):
        off = np.linalg.norm(a - np.diag(np.diag(a)))
        if off <= tol * scale:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if a[p, q] == 0.0:
                    continue
                theta = (a[q, q] - a[p, p]) / (2.0 * a[p, q])
                t = 1.0 if theta == 0.0 else np.sign(theta) / (abs(theta) + np.sqrt(1.0 + theta * theta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                ap = a[:, p].copy()
                a[:, p] = c * ap - s * a[:, q]
                a[:, q] = s * ap + c * a[:, q]
                ap = a[p, :].copy()
                a[p, :] = c * ap - s * a[q, :]
                a[q, :] = s * ap + c * a[q, :]
                vp = v[:, p].copy()
                v[:, p] = c * vp - s * v[:, q]
                v[:, q] = s * vp + c * v[:, q]
    w = np.diag(a).copy()
    order = np.argsort(-w, kind="stable")
    return w[order], v[:, order]


def fix_signs(u: np.ndarray, vt: np.ndarray = None):
    """Flip singular-vector pairs so the largest-|.| entry of each u_k is positive."""
    u = u.copy()
    idx = np.argmax(np.abs(u), axis=0)
    s = np.sign(u[idx, np.arange(u.shape[1])])
    s[s == 0] = 1.0
    u *= s[None, :]
    if vt is None:
        return u
    return u, vt * s[:, None]


def lstsq_qr(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Minimum-residual solution X of A X = B for full-column-rank A (m >= n).

    A = QR (Householder), X = R^{-1} Q^T B by back substitution.
    """
    q, r = householder_qr(a)
    rhs = q.T @ b
    n = r.shape[0]
    x = np.zeros((n,) + rhs.shape[1:])
    for i in range(n - 1, -1, -1):
        x[i] = (rhs[i] - r[i, i + 1:] @ x[i + 1:]) / r[i, i]
    return x
