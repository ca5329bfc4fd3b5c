"""Pins of the oracle's Householder QR, Jacobi SVD and least squares.

Each is checked against a LAPACK routine called through numpy (an independent
implementation), and against the defining properties (orthonormal Q, upper
triangular R with diag(R) >= 0, exact factorization), including exactly
rank-deficient inputs.
"""

import numpy as np
import pytest

from oracle import linalg as L


@pytest.mark.parametrize("m,l", [(10, 3), (64, 10), (200, 30), (33, 33)])
def test_householder_qr_matches_lapack_and_properties(m, l):
    y = np.random.default_rng(m * l).standard_normal((m, l))
    q, r = L.householder_qr(y)
    assert np.linalg.norm(q.T @ q - np.eye(l)) < 1e-13
    assert np.allclose(np.tril(r, -1), 0.0)
    assert np.all(np.diag(r) >= 0)
    np.testing.assert_allclose(q @ r, y, rtol=0, atol=1e-12 * np.linalg.norm(y))
    q2, r2 = np.linalg.qr(y)
    s = np.sign(np.diag(r2))
    np.testing.assert_allclose(q, q2 * s, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r, r2 * s[:, None], rtol=0, atol=1e-12 * np.linalg.norm(y))


def test_householder_qr_rank_deficient():
    rng = np.random.default_rng(5)
    y = rng.standard_normal((50, 4)) @ rng.standard_normal((4, 9))  # rank 4
    y[:, 6] = 0.0
    q, r = L.householder_qr(y)
    assert np.linalg.norm(q.T @ q - np.eye(9)) < 1e-13
    np.testing.assert_allclose(q @ r, y, rtol=0, atol=1e-12 * np.linalg.norm(y))
    # the range of the leading 4 columns of Q contains the range of Y
    p = q[:, :4] @ q[:, :4].T
    assert np.linalg.norm(y - p @ y) < 1e-12 * np.linalg.norm(y)


@pytest.mark.parametrize("m,n", [(12, 5), (5, 12), (40, 40), (100, 30)])
def test_jacobi_svd_matches_lapack(m, n):
    a = np.random.default_rng(m + 7 * n).standard_normal((m, n))
    u, s, vt = L.jacobi_svd(a)
    s_ref = np.linalg.svd(a, compute_uv=False)
    np.testing.assert_allclose(s, s_ref, rtol=1e-13, atol=1e-13 * s_ref[0])
    k = min(m, n)
    np.testing.assert_allclose((u[:, :k] * s[:k]) @ vt[:k], a, rtol=0, atol=1e-12 * s_ref[0])
    assert np.linalg.norm(u[:, :k].T @ u[:, :k] - np.eye(k)) < 1e-12
    assert np.linalg.norm(vt[:k] @ vt[:k].T - np.eye(k)) < 1e-12


def test_jacobi_svd_singular_vectors_match_lapack_up_to_sign():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((30, 8)) * np.logspace(0, -3, 8)[None, :]
    u, s, vt = L.jacobi_svd(a)
    u2, s2, vt2 = np.linalg.svd(a, full_matrices=False)
    ua, va = L.fix_signs(u, vt)
    ub, vb = L.fix_signs(u2, vt2)
    np.testing.assert_allclose(ua, ub, atol=1e-10)
    np.testing.assert_allclose(va, vb, atol=1e-10)


def test_lstsq_qr_matches_lapack():
    rng = np.random.default_rng(9)
    a = rng.standard_normal((75, 50))
    b = rng.standard_normal((75, 20))
    x = L.lstsq_qr(a, b)
    ref = np.linalg.lstsq(a, b, rcond=None)[0]
    np.testing.assert_allclose(x, ref, rtol=1e-10, atol=1e-11)
