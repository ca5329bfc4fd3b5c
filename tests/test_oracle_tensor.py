"""Pins of the oracle's unfolding / Khatri-Rao / TTM / MTTKRP (Sec. 2.1, Alg. 7).

* Brute force: nested loops over every index of the elementwise definitions
  Y_n[i_n, k] = sum_{i_j, j != n} X[i_1..i_d] prod_{j != n} Omega_j[i_j, k]
  and of the unfolding's column-index formula.
* numpy.einsum as an independent contraction path.
* The Gram identity (A kr B)^T (A kr B) = A^T A * B^T B and its d-factor form.
* The multilinear TTM identity Y_(i) = A_i X_(i) (A_d kron ... kron A_1, skip i).
* The closed form of the sketch of a Tucker tensor (mixed-product property):
  X = G x {U_j}  =>  Y_n = U_n G_(n) (kr_{j != n} U_j^T Omega_j).
"""

import itertools
import string

import numpy as np
import pytest

from oracle import tensor as T


def _rng(seed=0):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 4, 5), (4, 1, 3)])
def test_unfold_column_index_formula(dims):
    x = _rng(1).standard_normal(dims)
    d = len(dims)
    for n in range(d):
        xn = T.unfold(x, n)
        assert xn.shape == (dims[n], x.size // dims[n])
        for idx in itertools.product(*[range(k) for k in dims]):
            col, stride = 0, 1
            for j in range(d):
                if j == n:
                    continue
                col += idx[j] * stride
                stride *= dims[j]
            assert xn[idx[n], col] == x[idx]
        assert np.array_equal(T.fold(xn, n, dims), x)


def test_kron_and_khatri_rao_definitions():
    a = _rng(2).standard_normal((3, 4))
    b = _rng(3).standard_normal((5, 4))
    assert np.allclose(T.kron(a, b), np.kron(a, b), rtol=0, atol=0)
    kr = T.khatri_rao(a, b)
    for k in range(4):
        for i in range(3):
            for j in range(5):
                assert kr[i * 5 + j, k] == a[i, k] * b[j, k]


@pytest.mark.parametrize("nf", [2, 3, 4])
def test_khatri_rao_gram_identity(nf):
    rng = _rng(4 + nf)
    mats = [rng.standard_normal((rng.integers(2, 6), 7)) for _ in range(nf)]
    k = T.khatri_rao_list(mats)
    lhs = k.T @ k
    rhs = np.ones((7, 7))
    for m in mats:
        rhs = rhs * (m.T @ m)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dims,ell", [((3, 4, 5), 1), ((3, 4, 5), 3),
                                      ((2, 3, 4, 5), 2), ((5, 2, 3), 2)])
def test_mttkrp_brute_force_and_einsum(dims, ell):
    rng = _rng(11)
    x = rng.standard_normal(dims)
    om = [rng.standard_normal((n, ell)) for n in dims]
    d = len(dims)
    for n in range(d):
        y = T.mttkrp(x, om, n)
        # nested loops over every index of the elementwise definition
        ref = np.zeros((dims[n], ell))
        for idx in itertools.product(*[range(k) for k in dims]):
            for k in range(ell):
                w = 1.0
                for j in range(d):
                    if j != n:
                        w *= om[j][idx[j], k]
                ref[idx[n], k] += x[idx] * w
        np.testing.assert_allclose(y, ref, rtol=1e-13, atol=1e-13)
        # einsum: an independent contraction path
        letters = string.ascii_lowercase[:d]
        spec = letters + "".join("," + letters[j] + "z" for j in range(d) if j != n)
        spec += "->" + letters[n] + "z"
        ref2 = np.einsum(spec, x, *[om[j] for j in range(d) if j != n])
        np.testing.assert_allclose(y, ref2, rtol=1e-13, atol=1e-13)


def test_ttm_multilinear_identity():
    rng = _rng(21)
    dims = (3, 4, 5)
    x = rng.standard_normal(dims)
    a = [rng.standard_normal((r, n)) for r, n in zip((2, 3, 2), dims)]
    y = T.multi_ttm(x, a)
    for i in range(3):
        others = [a[j] for j in range(2, -1, -1) if j != i]
        kr = others[0]
        for m in others[1:]:
            kr = np.kron(kr, m)
        np.testing.assert_allclose(T.unfold(y, i), a[i] @ T.unfold(x, i) @ kr.T,
                                   rtol=1e-13, atol=1e-13)


def test_sketch_of_tucker_tensor_closed_form():
    rng = _rng(31)
    dims, core, ell = (6, 7, 8, 5), (2, 3, 2, 3), 4
    g = rng.standard_normal(core)
    u = [np.linalg.qr(rng.standard_normal((n, r)))[0] for n, r in zip(dims, core)]
    x = T.multi_ttm(g, u)
    om = [rng.standard_normal((n, ell)) for n in dims]
    for n in range(len(dims)):
        small = [u[j].T @ om[j] if j != n else None for j in range(len(dims))]
        closed = u[n] @ T.unfold(g, n) @ T.krp_except(small, n)
        np.testing.assert_allclose(T.mttkrp(x, om, n), closed, rtol=1e-12, atol=1e-12)


def test_frobenius_norm():
    x = _rng(5).standard_normal((4, 5, 6))
    assert T.frob(x) == pytest.approx(np.sqrt(sum(v * v for v in x.reshape(-1))), rel=1e-14)
