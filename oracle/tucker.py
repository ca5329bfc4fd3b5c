"""Tucker algorithms of Sec. 2.3 and Sec. 5.1, in FP64, by their printed steps.

  hosvd            Alg. 4 (HOSVD): leading left singular vectors of each X_(i)
  sthosvd          Alg. 5 (ST-HOSVD): same, on the partially truncated core
  rhosvd_krp       Alg. 7 (RHOSVD with Khatri-Rao products), fresh draws per mode
                   or (memo=True) the memoized variant RHOSVD-KRP-MEMO
  rsthosvd_krp     Alg. 8 (RSTHOSVD with Khatri-Rao products)
  truncate_core    rank-r truncation of a rank-l Tucker result by HOSVD of its
                   core (the analogue of Alg. 2's truncation step)
  rel_error        ||X - [G; Q_1..Q_d]||_F / ||X||_F, explicit reconstruction
  rel_error_slabs  the same, with the reconstruction formed one slab of the
                   last mode at a time (bounded memory for large X)

Draw ids of the sketching factors (contract with the device generator):
  memoized set: draw 0; fresh set of mode i (0-based): draw 1 + i;
  ST-HOSVD step i: draw 64 + i.  Factor index = mode index j.
"""

from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from . import philox
from .linalg import householder_qr, jacobi_svd
from .tensor import frob, multi_ttm, mttkrp, ttm, unfold, krp_except

MEMO_DRAW = 0
FRESH_DRAW_BASE = 1
STHOSVD_DRAW_BASE = 64


def _round(a: np.ndarray, mode: Optional[str]) -> np.ndarray:
    if mode is None or mode == "f64":
        return a
    if mode == "f32":
        return philox.round_to_f32(a)
    if mode == "bf16":
        return philox.round_to_bf16(a)
    raise ValueError(mode)


def leading_left_singular_vectors(m: np.ndarray, r: int) -> np.ndarray:
    """First r left singular vectors of m (numpy LAPACK SVD as the library step)."""
    u, _, _ = np.linalg.svd(m, full_matrices=False)
    return u[:, :r]


def hosvd(x: np.ndarray, ranks: Sequence[int]):
    """Alg. 4: Q_i = leading r_i left singular vectors of X_(i); G = X x {Q_i^T}."""
    qs = [leading_left_singular_vectors(unfold(x, i), r) for i, r in enumerate(ranks)]
    g = multi_ttm(x, [q.T for q in qs])
    return g, qs


def sthosvd(x: np.ndarray, ranks: Sequence[int]):
    """Alg. 5: for i = 1..d, Q_i from the current core G_(i), then G <- G x_i Q_i^T."""
    g = x
    qs = []
    for i, r in enumerate(ranks):
        q = leading_left_singular_vectors(unfold(g, i), r)
        g = ttm(g, q.T, i)
        qs.append(q)
    return g, qs


def memo_factors(seed: int, dims: Sequence[int], ell: int, omega_round=None):
    """The single factor set {Omega_j} (n_j x l) of RHOSVD-KRP-MEMO (Sec. 5.1)."""
    fs = philox.krp_factors(seed, MEMO_DRAW, dims, ell)
    return [_round(f, omega_round) for f in fs]


def fresh_factors(seed: int, dims: Sequence[int], mode: int, ell: int,
                  omega_round=None):
    """The d-1 factors Omega^(j) (n_j x l_i), j != i, drawn for mode i in Alg. 7."""
    fs = philox.krp_factors(seed, FRESH_DRAW_BASE + mode, dims, ell, skip=mode)
    return [None if f is None else _round(f, omega_round) for f in fs]


def rhosvd_krp(x: np.ndarray, ells: Sequence[int], seed: int, memo: bool = False,
               omega_round: Optional[str] = None):
    """Alg. 7 (RHOSVD-KRP); memo=True gives RHOSVD-KRP-MEMO.

    For each mode i: draw the factors (fresh: d-1 new n_j x l_i matrices; memo:
    the shared set, of which the first l_i columns are used), sketch
    Y_i = X_(i) (Omega^(d) kr ... kr Omega^(i+1) kr Omega^(i-1) kr ... kr Omega^(1)),
    orthonormalise Y_i = Q_i R.  Then G = X x_1 Q_1^T ... x_d Q_d^T.
    Returns dict(G, Q, Y, omega).
    """
    d = x.ndim
    dims = x.shape
    ells = list(ells)
    shared = memo_factors(seed, dims, max(ells), omega_round) if memo else None
    qs: List[np.ndarray] = []
    ys: List[np.ndarray] = []
    oms = []
    for i in range(d):
        if memo:
            om = [f[:, :ells[i]] if j != i else None for j, f in enumerate(shared)]
        else:
            om = fresh_factors(seed, dims, i, ells[i], omega_round)
        y = mttkrp(x, om, i)
        q, _ = householder_qr(y)
        ys.append(y)
        qs.append(q)
        oms.append(om)
    g = multi_ttm(x, [q.T for q in qs])
    return {"G": g, "Q": qs, "Y": ys, "omega": oms}


def sthosvd_factors(seed: int, rows: Sequence[int], step: int, ell: int,
                    omega_round=None):
    """Factors of ST-HOSVD step i (Alg. 8): Omega^(j) is rows[j] x l_i, j != i."""
    fs = philox.krp_factors(seed, STHOSVD_DRAW_BASE + step, rows, ell, skip=step)
    return [None if f is None else _round(f, omega_round) for f in fs]


def rsthosvd_krp(x: np.ndarray, ells: Sequence[int], seed: int,
                 omega_round: Optional[str] = None):
    """Alg. 8 (RSTHOSVD-KRP), modes processed in the order 1..d.

    Step i: the current core G has sides (l_1..l_{i-1}, n_i..n_d); draw
    Omega^(j) in R^{l_j x l_i} (j < i) and R^{n_j x l_i} (j > i); sketch
    Y_i = G_(i) K_i; Q_i R = Y_i; G <- G x_i Q_i^T.
    Returns dict(G, Q, Y, omega, cores) with the partial cores G^(0..d).
    """
    d = x.ndim
    g = x
    qs, ys, oms, cores = [], [], [], [x]
    for i in range(d):
        om = sthosvd_factors(seed, g.shape, i, ells[i], omega_round)
        y = mttkrp(g, om, i)
        q, _ = householder_qr(y)
        g = ttm(g, q.T, i)
        qs.append(q)
        ys.append(y)
        oms.append(om)
        cores.append(g)
    return {"G": g, "Q": qs, "Y": ys, "omega": oms, "cores": cores}


def truncate_core(g: np.ndarray, qs: Sequence[np.ndarray], ranks: Sequence[int]):
    """Rank-(r_1..r_d) truncation of [G; Q_1..Q_d] through an HOSVD of the core.

    U_i = leading r_i left singular vectors of G_(i) (one-sided Jacobi SVD);
    G <- G x_1 U_1^T ... x_d U_d^T and Q_i <- Q_i U_i.  Because every Q_i has
    orthonormal columns this equals the HOSVD (Alg. 4) of the rank-l
    approximation itself, computed on the small core.
    """
    us = []
    for i, r in enumerate(ranks):
        u, _, _ = jacobi_svd(unfold(g, i))
        us.append(u[:, :r])
    g2 = multi_ttm(g, [u.T for u in us])
    return g2, [q @ u for q, u in zip(qs, us)]


def reconstruct(g: np.ndarray, qs: Sequence[np.ndarray]) -> np.ndarray:
    """X_hat = G x_1 Q_1 ... x_d Q_d."""
    return multi_ttm(g, qs)


def rel_error(x: np.ndarray, g: np.ndarray, qs: Sequence[np.ndarray]) -> float:
    """||X - X_hat||_F / ||X||_F with the reconstruction formed explicitly."""
    return frob(x - reconstruct(g, qs)) / frob(x)


def rel_error_slabs(x: np.ndarray, g: np.ndarray, qs: Sequence[np.ndarray],
                    slab: int = 64) -> float:
    """rel_error with X_hat formed slab by slab along the last mode.

    X_hat[..., t] depends on row t of Q_d only, so the slab t0 <= t < t1 of the
    reconstruction is G x_1 Q_1 ... x_{d-1} Q_{d-1} x_d Q_d[t0:t1]; the squared
    residuals of the slabs add up to ||X - X_hat||_F^2.  Only one slab of
    X_hat is held at a time.
    """
    n_d = x.shape[-1]
    num = 0.0
    for t0 in range(0, n_d, slab):
        t1 = min(n_d, t0 + slab)
        part = reconstruct(g, list(qs[:-1]) + [qs[-1][t0:t1]])
        num += float(np.sum(np.square(x[..., t0:t1] - part, dtype=np.float64)))
    nx = frob(x)
    return float(np.sqrt(num)) / nx if nx > 0 else 0.0


def mttkrp_rows(x: np.ndarray, omegas, n: int, rows) -> np.ndarray:
    """Selected rows of Y_n = X_(n) K_n (explicit KRP), for sampled parity checks."""
    return unfold(x, n)[np.asarray(rows)] @ krp_except(omegas, n)


# ---- random-number counts (Table 1 and the text after it) --------------------

def rng_count_rhosvd_krp(dims: Sequence[int], ells: Sequence[int]) -> int:
    """Normals drawn by Alg. 7: sum_i sum_{j != i} n_j l_i."""
    d = len(dims)
    return sum(dims[j] * ells[i] for i in range(d) for j in range(d) if j != i)


def rng_count_memo(dims: Sequence[int], ell: int) -> int:
    """Normals drawn by the memoized variant: one factor per mode, sum_j n_j l."""
    return sum(int(n) * ell for n in dims)


def rng_count_rsthosvd_krp(dims: Sequence[int], ells: Sequence[int]) -> int:
    """Normals drawn by Alg. 8: step i draws l_j x l_i (j < i) and n_j x l_i (j > i)."""
    d = len(dims)
    total = 0
    for i in range(d):
        for j in range(d):
            if j < i:
                total += ells[j] * ells[i]
            elif j > i:
                total += dims[j] * ells[i]
    return total
