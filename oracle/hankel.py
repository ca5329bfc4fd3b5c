"""Block-structured matrices and Alg. 6 (single-pass randomized SVD for them), FP64.

M = sum_j E_j kron M_j with 0/1 patterns E_j (p x q) and m x n blocks M_j
(Sec. 4).  For the block Hankel matrix of Sec. 4.2, E_k (s x s) has ones where
i + j - 1 = k, so block (i, j) (1-based) is H_{i+j-1}, k = 1..2s-1.

The oracle forms M, Omega = Omega^(1) kr Omega^(2) and Psi = Psi^(1) kr Psi^(2)
explicitly and multiplies; the structured identity of Eq. (4.1),
M Omega = sum_j (E_j Omega^(1)) kr (M_j Omega^(2)), is what the CUDA path
computes instead, and the tests pin the two against each other.

Factor draws (Philox contract): Omega^(1) = factor 0, Omega^(2) = factor 1 on
stream tag 0; Psi^(1) = factor 0, Psi^(2) = factor 1 on tag 1; draw id 0.
"""

from __future__ import annotations

import numpy as np

from . import philox
from .linalg import householder_qr, jacobi_eig, jacobi_svd, lstsq_qr
from .tensor import khatri_rao, khatri_rao_list


def block_hankel(blocks: np.ndarray) -> np.ndarray:
    """Explicit (m s) x (n s) block Hankel matrix from blocks (m, n, 2s-1)."""
    m, n, nb = blocks.shape
    s = (nb + 1) // 2
    if nb != 2 * s - 1:
        raise ValueError("a block Hankel needs 2s-1 blocks")
    h = np.zeros((m * s, n * s))
    for i in range(s):
        for j in range(s):
            h[i * m:(i + 1) * m, j * n:(j + 1) * n] = blocks[:, :, i + j]
    return h


def hankel_pattern(s: int, k: int) -> np.ndarray:
    """E_k in R^{s x s}: ones where i + j - 1 = k (1-based), zeros elsewhere."""
    e = np.zeros((s, s))
    for i in range(s):
        j = k - 1 - i  # 0-based: i + j = k - 1
        if 0 <= j < s:
            e[i, j] = 1.0
    return e


def structured_sketch(blocks: np.ndarray, om1: np.ndarray, om2: np.ndarray,
                      transpose: bool = False) -> np.ndarray:
    """sum_k (E_k Omega^(1)) kr (H_k Omega^(2)) of Eq. (4.1).

    With transpose=True: sum_k (E_k^T Psi^(1)) kr (H_k^T Psi^(2)), the row sketch
    M^T Psi of Alg. 6.
    """
    m, n, nb = blocks.shape
    s = (nb + 1) // 2
    out = 0.0
    for k in range(1, nb + 1):
        e = hankel_pattern(s, k)
        hk = blocks[:, :, k - 1]
        if transpose:
            e, hk = e.T, hk.T
        out = out + khatri_rao(e @ om1, hk @ om2)
    return out


def sketch_factors(seed: int, s: int, m: int, n: int, ell_r: int, ell_l: int,
                   omega_round=None):
    """(Omega^(1) s x l_r, Omega^(2) n x l_r, Psi^(1) s x l_l, Psi^(2) m x l_l)."""
    o1 = philox.gaussian_factor(seed, 0, 0, philox.TAG_OMEGA, s, ell_r)
    o2 = philox.gaussian_factor(seed, 1, 0, philox.TAG_OMEGA, n, ell_r)
    p1 = philox.gaussian_factor(seed, 0, 0, philox.TAG_PSI, s, ell_l)
    p2 = philox.gaussian_factor(seed, 1, 0, philox.TAG_PSI, m, ell_l)
    if omega_round == "f32":
        o1, o2, p1, p2 = (philox.round_to_f32(a) for a in (o1, o2, p1, p2))
    elif omega_round == "bf16":
        o1, o2, p1, p2 = (philox.round_to_bf16(a) for a in (o1, o2, p1, p2))
    return o1, o2, p1, p2


def single_pass_svd(blocks: np.ndarray, r: int, ell_r: int, ell_l: int, seed: int,
                    omega_round=None):
    """Alg. 6 on the explicit block Hankel matrix.

    1. Omega = Omega^(1) kr Omega^(2), Psi = Psi^(1) kr Psi^(2)
    2. Y = M Omega, Z = M^T Psi
    3. Y = Q R (Householder)
    4. W = (Psi^T Q)^+ Z^T (least squares)
    5. W = U_W Sigma V^T
    6. U = Q U_W
    7. return U[:, :r], Sigma[:r], V[:, :r]
    Also returns the intermediates for tests.
    """
    m, n, nb = blocks.shape
    s = (nb + 1) // 2
    o1, o2, p1, p2 = sketch_factors(seed, s, m, n, ell_r, ell_l, omega_round)
    h = block_hankel(blocks)
    omega = khatri_rao(o1, o2)
    psi = khatri_rao(p1, p2)
    y = h @ omega
    z = h.T @ psi
    q, _ = householder_qr(y)
    w = lstsq_qr(psi.T @ q, z.T)
    uw, sig, vt = jacobi_svd(w)
    u = q @ uw
    return {"U": u[:, :r], "S": sig[:r], "V": vt[:r].T, "Y": y, "Z": z, "Q": q,
            "W": w, "factors": (o1, o2, p1, p2), "H": h}


# Reading of the pseudoinverse in the Nystrom approximation: eigenvalues of
# Omega^T M Omega at or below NYS_RCOND times the largest are treated as zero.
NYS_RCOND = 1e-6


def nystrom(blocks: np.ndarray, r: int, ell: int, seed: int, rcond: float = NYS_RCOND,
            omega_round=None):
    """Nystrom approximation of a symmetric positive semidefinite block Hankel
    matrix M (Sec. 4.1, the remark after Alg. 6):

        M_nys = (M Omega) (Omega^T M Omega)^+ (M Omega)^T,  Omega = Omega^(1) kr Omega^(2),

    with Omega the column-sketch factors of Alg. 6 (s x l and m x l, tag 0,
    draw 0).  Steps, on the explicit matrices:
    1. Y = M Omega
    2. C = Omega^T Y (symmetrised), C = V diag(c) V^T (two-sided Jacobi)
    3. the pseudoinverse keeps c_i > rcond * c_1: M_nys = F F^T with
       F = Y V_k diag(c_k^{-1/2})
    4. F = U Sigma W^T (one-sided Jacobi SVD), so M_nys = U Sigma^2 U^T
    Returns U[:, :r] and Lambda = Sigma[:r]^2 (zero-padded when fewer than r
    eigenvalues are kept), with M_nys, Y, C and the kept count for tests.
    """
    m, n, nb = blocks.shape
    if m != n:
        raise ValueError("the Nystrom approximation needs square blocks")
    s = (nb + 1) // 2
    o1, o2, _, _ = sketch_factors(seed, s, m, n, ell, 1, omega_round)
    h = block_hankel(blocks)
    omega = khatri_rao(o1, o2)
    y = h @ omega
    c = omega.T @ y
    c = 0.5 * (c + c.T)
    cv, vv = jacobi_eig(c)
    keep = cv > rcond * cv[0] if cv[0] > 0.0 else np.zeros(ell, dtype=bool)
    f = (y @ vv[:, keep]) / np.sqrt(cv[keep])
    u = np.zeros((m * s, r))
    lam = np.zeros(r)
    k = int(keep.sum())
    if k:
        uf, sig, _ = jacobi_svd(f)
        u[:, :min(r, k)] = uf[:, :r]
        lam[:min(r, k)] = sig[:r] ** 2
    return {"U": u, "L": lam, "M": f @ f.T, "Y": y, "C": c, "kept": k, "H": h}


def era_realization(blocks: np.ndarray, u: np.ndarray, sig: np.ndarray,
                    v: np.ndarray) -> np.ndarray:
    """State matrix of the eigensystem realization built from a rank-r SVD of
    the block Hankel matrix (the use Sec. 4.2 makes of Alg. 6).

    With H = U S V^T, the observability factor is O = U S^{1/2} and the
    controllability factor is G = S^{1/2} V^T.  The shifted block Hankel
    matrix H_up has h_{i+j} in block (i, j), for i = 1..s-1 and j = 1..s, so
    it uses blocks 2..2s-1 only.  It equals O_top A G, where O_top is the
    first (s-1) m rows of O.  Hence A = O_top^+ H_up G^+, with
    G^+ = V S^{-1/2}.  A is returned up to a similarity transform, so its
    eigenvalues are those of the system.
    """
    m, n, nb = blocks.shape
    s = (nb + 1) // 2
    h_up = np.zeros(((s - 1) * m, s * n))
    for i in range(s - 1):
        for j in range(s):
            h_up[i * m:(i + 1) * m, j * n:(j + 1) * n] = blocks[:, :, i + j + 1]
    sq = np.sqrt(sig)
    o_top = u[:(s - 1) * m] * sq
    g_pinv = v / sq
    return np.linalg.lstsq(o_top, h_up @ g_pinv, rcond=None)[0]


def hausdorff(a: np.ndarray, b: np.ndarray) -> float:
    """Hausdorff distance between two finite sets of complex numbers."""
    d = np.abs(np.asarray(a)[:, None] - np.asarray(b)[None, :])
    return float(max(d.min(axis=1).max(), d.min(axis=0).max()))


def rng_count_block(m: int, n: int, p: int, q: int, ell_r: int, ell_l: int) -> int:
    """Normals drawn by Alg. 6 with KRP sketches: (n+q) l_r + (m+p) l_l (Sec. 4.1)."""
    return (n + q) * ell_r + (m + p) * ell_l


def rng_count_block_gauss(m: int, n: int, p: int, q: int, ell_r: int,
                          ell_l: int) -> int:
    """Normals for the same algorithm with dense Gaussian sketches: nq l_r + mp l_l."""
    return n * q * ell_r + m * p * ell_l


# ---- two-level block Hankel matrices (Sec. 4.3, multilevel structure) ----
#
# M = sum_{k1, k2} E_{k1} kron E_{k2} kron H_{k1,k2}: s1 x s1 blocks, block
# (i1, j1) itself an s2 x s2 block Hankel matrix whose block (i2, j2) is
# H_{i1+j1, i2+j2} (0-based), each m x n.  blocks has shape
# (m, n, 2 s1 - 1, 2 s2 - 1); row index a + m (i2 + s2 i1), column index
# b + n (j2 + s2 j1).  Factor draws: Omega = Omega^(1) kr Omega^(2) kr
# Omega^(3) (s1, s2, n rows: factors 0, 1, 2 on tag 0), Psi likewise with
# (s1, s2, m) rows on tag 1; draw id 0.


def block_hankel2(blocks: np.ndarray) -> np.ndarray:
    """Explicit (m s1 s2) x (n s1 s2) two-level block Hankel matrix."""
    m, n, nb1, nb2 = blocks.shape
    s1, s2 = (nb1 + 1) // 2, (nb2 + 1) // 2
    if nb1 != 2 * s1 - 1 or nb2 != 2 * s2 - 1:
        raise ValueError("a two-level block Hankel needs (2 s1 - 1) x (2 s2 - 1) blocks")
    h = np.zeros((m * s1 * s2, n * s1 * s2))
    for i1 in range(s1):
        for j1 in range(s1):
            for i2 in range(s2):
                for j2 in range(s2):
                    r0 = m * (i2 + s2 * i1)
                    c0 = n * (j2 + s2 * j1)
                    h[r0:r0 + m, c0:c0 + n] = blocks[:, :, i1 + j1, i2 + j2]
    return h


def structured_sketch2(blocks: np.ndarray, o1: np.ndarray, o2: np.ndarray, o3: np.ndarray,
                       transpose: bool = False) -> np.ndarray:
    """sum_{k1,k2} (E_{k1} O1) kr (E_{k2} O2) kr (H_{k1,k2} O3), the two-level
    form of Eq. (4.1) (mixed-product property of the Kronecker and
    Khatri-Rao products); with transpose=True the blocks enter transposed
    (the row sketch M^T Psi)."""
    m, n, nb1, nb2 = blocks.shape
    s1, s2 = (nb1 + 1) // 2, (nb2 + 1) // 2
    out = 0.0
    for k1 in range(1, nb1 + 1):
        e1 = hankel_pattern(s1, k1)
        for k2 in range(1, nb2 + 1):
            e2 = hankel_pattern(s2, k2)
            hk = blocks[:, :, k1 - 1, k2 - 1]
            if transpose:
                hk = hk.T
            out = out + khatri_rao_list([e1.T @ o1 if transpose else e1 @ o1,
                                         e2.T @ o2 if transpose else e2 @ o2, hk @ o3])
    return out


def sketch_factors2(seed: int, s1: int, s2: int, m: int, n: int, ell_r: int, ell_l: int,
                    omega_round=None):
    """(Omega^(1..3), Psi^(1..3)): s1, s2, n rows x l_r and s1, s2, m rows x l_l."""
    om = [philox.gaussian_factor(seed, f, 0, philox.TAG_OMEGA, rows, ell_r)
          for f, rows in enumerate((s1, s2, n))]
    ps = [philox.gaussian_factor(seed, f, 0, philox.TAG_PSI, rows, ell_l)
          for f, rows in enumerate((s1, s2, m))]
    if omega_round == "f32":
        om, ps = [philox.round_to_f32(a) for a in om], [philox.round_to_f32(a) for a in ps]
    elif omega_round == "bf16":
        om, ps = [philox.round_to_bf16(a) for a in om], [philox.round_to_bf16(a) for a in ps]
    return om, ps


def single_pass_svd2(blocks: np.ndarray, r: int, ell_r: int, ell_l: int, seed: int,
                     omega_round=None):
    """Alg. 6 on the explicit two-level block Hankel matrix, with
    Omega = Omega^(1) kr Omega^(2) kr Omega^(3) and Psi likewise:
    Y = M Omega, Z = M^T Psi, Y = QR, W = (Psi^T Q)^+ Z^T, W = U_W S V^T,
    U = Q U_W; returns U[:, :r], S[:r], V[:, :r] and the intermediates."""
    m, n, nb1, nb2 = blocks.shape
    s1, s2 = (nb1 + 1) // 2, (nb2 + 1) // 2
    om, ps = sketch_factors2(seed, s1, s2, m, n, ell_r, ell_l, omega_round)
    h = block_hankel2(blocks)
    omega = khatri_rao_list(om)
    psi = khatri_rao_list(ps)
    y = h @ omega
    z = h.T @ psi
    q, _ = householder_qr(y)
    w = lstsq_qr(psi.T @ q, z.T)
    uw, sig, vt = jacobi_svd(w)
    u = q @ uw
    return {"U": u[:, :r], "S": sig[:r], "V": vt[:r].T, "Y": y, "Z": z, "Q": q, "W": w,
            "factors": (om, ps), "H": h}
