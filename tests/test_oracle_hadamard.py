"""Pins for the Hadamard-product recompression.

* The structure the CUDA path uses: the elementwise product of two Tucker
  tensors is a Tucker tensor with the Kronecker core G (x) H (index
  c_j = a_j + r_j b_j) and the row-wise Khatri-Rao (face-splitting) factors
  W_j[i, c_j] = U_j[i, a_j] V_j[i, b_j]; built here with numpy kron and
  elementwise products, independent of the oracle's explicit product.
* The sketch of Z through that structure: Z_(n) K_n = W_n MTTKRP(G (x) H,
  {W_j^T Omega_j}) (mixed-product property), against the explicit MTTKRP.
* Exact recovery: with l >= the product's multilinear rank (r_j s_j) the
  recompression reproduces Z.
"""

import numpy as np

from oracle import hadamard as HD, tensor as T, tucker as TK
from synth import haar


def _pair(dims, r, s, seed):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(r)
    h = rng.standard_normal(s)
    us = [haar(n, k, rng) for n, k in zip(dims, r)]
    vs = [haar(n, k, rng) for n, k in zip(dims, s)]
    return g, us, h, vs


def _kron_core(g, h):
    # C[c_1..c_d], c_j = a_j + r_j b_j: G's index fastest within each pair
    d = g.ndim
    c = np.multiply.outer(g, h)  # axes a_1..a_d, b_1..b_d
    perm = [x for j in range(d) for x in (j, d + j)]
    c = np.transpose(c, perm)    # a_1, b_1, a_2, b_2, ...
    shape = [g.shape[j] * h.shape[j] for j in range(d)]
    return np.reshape(c, shape, order="F")


def _face_split(u, v):
    return np.einsum("ia,ib->iab", u, v).reshape(u.shape[0], -1, order="F")


def test_product_is_kronecker_tucker():
    dims, r, s = (9, 8, 7), (3, 2, 3), (2, 3, 2)
    g, us, h, vs = _pair(dims, r, s, 1)
    z = HD.hadamard_of_tucker(g, us, h, vs)
    x = TK.reconstruct(g, us) * TK.reconstruct(h, vs)
    assert np.array_equal(z, x)
    c = _kron_core(g, h)
    ws = [_face_split(u, v) for u, v in zip(us, vs)]
    assert np.linalg.norm(TK.reconstruct(c, ws) - z) <= 1e-12 * np.linalg.norm(z)


def test_structured_sketch_of_the_product():
    dims, r, s, ell = (9, 8, 7), (3, 2, 3), (2, 3, 2), 5
    g, us, h, vs = _pair(dims, r, s, 2)
    z = HD.hadamard_of_tucker(g, us, h, vs)
    om = TK.memo_factors(4, dims, ell)
    c = _kron_core(g, h)
    ws = [_face_split(u, v) for u, v in zip(us, vs)]
    ps = [w.T @ o for w, o in zip(ws, om)]
    for n in range(3):
        y = T.mttkrp(z, om, n)
        m = T.mttkrp(c, ps, n)
        assert np.linalg.norm(ws[n] @ m - y) <= 1e-12 * np.linalg.norm(y)


def test_exact_recovery_at_full_product_rank():
    dims, r, s = (12, 11, 10), (2, 2, 2), (2, 2, 2)
    g, us, h, vs = _pair(dims, r, s, 3)
    out = HD.rhosvd_krp_hadamard(g, us, h, vs, 6, seed=5)
    assert out["rel_error"] <= 1e-10
