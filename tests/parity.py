"""Comparison of error values (P3) and reconstructions (P2) between the
library and the FP64 oracle, with the tolerance derived from the arithmetic.

P3 compares e = ||X - X_hat||_F / ||X||_F as the library reports it (e_gpu)
with the oracle's value (e_ora).  Two things separate them:

  eta   = ||X_hat_gpu - X_hat_ora||_F / ||X||_F, the distance between the two
          approximations (P2; measured in the test from the returned core and
          factors);
  rho   = the evaluation error of the library's residual pass, which rebuilds
          X_hat in FP32 (or from BF16 hi/lo pairs) and sums (x - x_hat)^2.

With e_self the exact (FP64, oracle-evaluated) relative error of the
library's own (G, Q), the triangle inequality gives
  |e_gpu - e_ora| <= |e_gpu - e_self| + |e_self - e_ora| <= rho + eta.
The printed P3 bound 1e-5 max(e_ora, 1e-6) is reachable only where
e >> eta + rho; below that the FP32 form cannot resolve e to 1e-5 relative,
because FP32 rounding of the sketch moves the captured subspace (eta) and FP32
rounding of x_hat moves the evaluated norm (rho).  The tests therefore assert
  (a) |e_gpu - e_self| <= 1e-5 max(e_self, 1e-6) + rho
  (b) |e_gpu - e_ora|  <= 1e-5 max(e_ora, 1e-6) + eta + rho
with eta measured (it is itself bounded by P2) and rho from the rounding model
below.  A returned residual of 0, or one off by more than eta + rho, fails.

Rounding model for rho.  The residual pass perturbs the reconstruction by
delta = sum_j delta_j, one term per expansion stage j (FP32 storage of factor
j, c_j FP32 accumulations, one rounding of the stage output), each of relative
RMS at most unit * sqrt(c_j + 2) (independent roundings of relative size
<= unit add in quadrature), so s = ||delta||_F / ||X||_F
<= unit * sqrt(sum_j (c_j + 2)) * ||X_hat||_F / ||X||_F.  Then
  e_gpu^2 ||X||^2 = ||r - delta||^2 = ||r||^2 - 2 <r, delta> + ||delta||^2,
so |e_gpu - e_self| <= |<r, delta>| / (e ||X||^2) + s^2 / (2 e).  delta is
built from at least min_j n_j independent roundings (the entries of a factor
column), so its cosine with the fixed residual r is at most 4 / sqrt(min_j
n_j) (four standard deviations): rho = 4 s / sqrt(min_j n_j) + s^2 / (2 e).
unit is 2^-24 for FP32 operands and 2^-16 for BF16 hi/lo pairs (the pair
represents a value to 2^-18 and the MMAs drop the lo x lo products, 2^-18
each).  The FP32 form expands modes 2..d with FP32 FMAs (unit 2^-24) and may
run the mode-1 stage on the tensor cores as three TF32 products of FP32
operands split as v = v_h + v_l (v_h: v with its low 13 mantissa bits
cleared, v_l exact in FP32): the MMA reads v_l truncated to TF32 (error
< 2^-10 |v_l| < 2^-20 |v|, for each of the two operands) and the dropped
v_l w_l term is < 2^-20 |v w|, so a product is off by < 3 * 2^-20 relative
in the worst case; unit1 = 2^-18 for that stage (U_TF32_PAIR), above that
worst case as the BF16 pair's unit is above its own (tests/test_tf32_split.py
pins the three error terms on emulated TF32 arithmetic).
"""

from __future__ import annotations

import math
from typing import Sequence

import numpy as np

U_F32 = 2.0 ** -24
U_BF16_PAIR = 2.0 ** -16
U_TF32_PAIR = 2.0 ** -18


def eval_bound(cols: Sequence[int], dims: Sequence[int], xhat_over_x: float, e_self: float,
               unit: float = U_F32, unit1: float | None = None) -> float:
    """rho of the module docstring; unit1 is the unit of the mode-1 stage
    (cols[0]) where it differs from the others'."""
    u1 = unit if unit1 is None else unit1
    cs = [int(c) for c in cols]
    s = math.sqrt(u1 * u1 * (cs[0] + 2) + unit * unit * sum(c + 2 for c in cs[1:])) * xhat_over_x
    if s == 0.0:
        return 0.0
    return 4.0 * s / math.sqrt(min(int(n) for n in dims)) + s * s / (2.0 * max(e_self, s))


def check_error_value(e_gpu: float, e_ora: float, e_self: float, eta: float, rho: float,
                      what: str = "") -> None:
    """Assert (a) and (b) of the module docstring."""
    d_self = abs(e_gpu - e_self)
    d_ora = abs(e_gpu - e_ora)
    b_self = 1e-5 * max(e_self, 1e-6) + rho
    b_ora = 1e-5 * max(e_ora, 1e-6) + eta + rho
    assert d_self <= b_self, (what, "e_gpu vs exact error of the library's own result",
                              e_gpu, e_self, d_self, b_self)
    assert d_ora <= b_ora, (what, "e_gpu vs oracle", e_gpu, e_ora, d_ora, b_ora, eta, rho)


def recon_distance(g1: np.ndarray, q1: Sequence[np.ndarray], g2: np.ndarray,
                   q2: Sequence[np.ndarray]) -> float:
    """||G1 x {Q1_i} - G2 x {Q2_i}||_F without forming either reconstruction:
    with B_i an orthonormal basis of [Q1_i, Q2_i] (Householder QR), both
    reconstructions lie in the span of B_1 (x) ... (x) B_d, where the map is
    an isometry, so the distance equals that of the small tensors
    G1 x {B_i^T Q1_i} and G2 x {B_i^T Q2_i}."""
    a, b = g1, g2
    for i, (u, v) in enumerate(zip(q1, q2)):
        basis, _ = np.linalg.qr(np.concatenate([u, v], axis=1))
        a = np.moveaxis(np.tensordot(basis.T @ u, a, axes=(1, i)), 0, i)
        b = np.moveaxis(np.tensordot(basis.T @ v, b, axes=(1, i)), 0, i)
    return float(np.linalg.norm(a - b))


def projector_distance(qa: np.ndarray, qb: np.ndarray) -> float:
    """||Qa Qa^T - Qb Qb^T||_F / sqrt(r) for equal-rank orthonormal Qa, Qb,
    as sqrt(2) ||(I - Qb Qb^T) Qa||_F / sqrt(r) (no n x n matrix formed)."""
    r = qa.shape[1]
    return float(math.sqrt(2.0) * np.linalg.norm(qa - qb @ (qb.T @ qa)) / math.sqrt(r))
