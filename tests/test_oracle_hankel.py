"""Pins of the oracle's block-Hankel construction and Alg. 6 (Sec. 4).

* The block Hankel matrix equals sum_k E_k kron H_k with the 0/1 patterns E_k
  of Sec. 4.2, built from explicit Kronecker products.
* Eq. (4.1): M (Omega1 kr Omega2) = sum_k (E_k Omega1) kr (H_k Omega2), and the
  mirror identity for M^T (Psi1 kr Psi2).
* Exact-rank input: the single-pass approximation reproduces H (the two-sided
  sketch is exact when rank(M) <= l_r, Sec. 4.4) and its singular values match
  LAPACK's.
* Random-number counts: the shares printed in Sec. 4.2 (golden fixture).
"""

import math
import os

import numpy as np
import pytest

from oracle import hankel as HK
from oracle import tensor as T
from synth import HankelSpec, markov_parameters
from synth.hankel import system_matrices

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_spec(order=6, m=3, n=2, s=9, seed=5):
    return HankelSpec("t", order, m, n, s, 0.9, seed, r=order, ell_r=order + 4,
                      ell_l=int(math.ceil(1.5 * (order + 4))))


def test_block_hankel_is_sum_of_kronecker_patterns():
    sp = small_spec()
    blocks = markov_parameters(sp)
    h = HK.block_hankel(blocks)
    ref = sum(T.kron(HK.hankel_pattern(sp.s, k), blocks[:, :, k - 1])
              for k in range(1, sp.nblocks + 1))
    assert np.array_equal(h, ref)
    # Hankel: block (i, j) depends on i + j only
    assert np.array_equal(h[:sp.m, sp.n:2 * sp.n], h[sp.m:2 * sp.m, :sp.n])


def test_markov_parameters_definition():
    sp = small_spec()
    a, b, c, eig = system_matrices(sp)
    blocks = markov_parameters(sp)
    np.testing.assert_allclose(blocks[:, :, 0], c @ b, rtol=1e-14)
    np.testing.assert_allclose(blocks[:, :, 4], c @ np.linalg.matrix_power(a, 4) @ b,
                               rtol=1e-12, atol=1e-14)
    ev = np.linalg.eigvals(a)
    assert np.max(np.abs(ev)) <= sp.radius + 1e-12
    for e in eig:
        assert np.min(np.abs(ev - e)) < 1e-10


def test_structured_sketch_identity_eq_4_1():
    sp = small_spec()
    blocks = markov_parameters(sp)
    h = HK.block_hankel(blocks)
    rng = np.random.default_rng(1)
    o1, o2 = rng.standard_normal((sp.s, 5)), rng.standard_normal((sp.n, 5))
    p1, p2 = rng.standard_normal((sp.s, 7)), rng.standard_normal((sp.m, 7))
    np.testing.assert_allclose(HK.structured_sketch(blocks, o1, o2),
                               h @ T.khatri_rao(o1, o2), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(HK.structured_sketch(blocks, p1, p2, transpose=True),
                               h.T @ T.khatri_rao(p1, p2), rtol=1e-12, atol=1e-13)


def test_single_pass_exact_rank_recovery():
    sp = small_spec(order=6, m=3, n=2, s=12, seed=9)
    blocks = markov_parameters(sp)
    res = HK.single_pass_svd(blocks, sp.r, sp.ell_r, sp.ell_l, seed=0)
    h = res["H"]
    approx = (res["U"] * res["S"]) @ res["V"].T
    assert np.linalg.norm(h - approx) <= 1e-10 * np.linalg.norm(h)
    s_ref = np.linalg.svd(h, compute_uv=False)[:sp.r]
    np.testing.assert_allclose(res["S"], s_ref, rtol=1e-8)
    assert np.linalg.norm(res["U"].T @ res["U"] - np.eye(sp.r)) < 1e-12
    assert np.linalg.norm(res["V"].T @ res["V"] - np.eye(sp.r)) < 1e-12


def test_era_from_single_pass_recovers_the_system_eigenvalues():
    """End-to-end pin of Alg. 6 through ERA.  The data come from a known
    order-8 system, so the eigenvalues of the realized state matrix are fixed
    by construction.  Alg. 6's rank-r factors must reproduce them up to
    rounding.  With r one below the order they must not."""
    sp = HankelSpec("era", 8, 3, 3, 14, 0.9, 21, r=8, ell_r=12, ell_l=18)
    blocks = markov_parameters(sp)
    _, _, _, eig = system_matrices(sp)
    res = HK.single_pass_svd(blocks, sp.r, sp.ell_r, sp.ell_l, seed=3)
    a_hat = HK.era_realization(blocks, res["U"], res["S"], res["V"])
    assert a_hat.shape == (8, 8)
    assert HK.hausdorff(np.linalg.eigvals(a_hat), eig) <= 1e-11
    # the exact SVD gives the same realization spectrum (a check of era_realization
    # that does not depend on the sketch)
    uh, sh, vth = np.linalg.svd(res["H"])
    a_ref = HK.era_realization(blocks, uh[:, :8], sh[:8], vth[:8].T)
    assert HK.hausdorff(np.linalg.eigvals(a_ref), eig) <= 1e-11
    # truncating below the order loses an eigenvalue pair's worth of the spectrum
    res7 = HK.single_pass_svd(blocks, 7, sp.ell_r, sp.ell_l, seed=3)
    a7 = HK.era_realization(blocks, res7["U"], res7["S"], res7["V"])
    assert HK.hausdorff(np.linalg.eigvals(a7), eig) > 1e-3


def test_hausdorff_distance():
    a = np.array([0.0, 1.0 + 1.0j])
    assert HK.hausdorff(a, a) == 0.0
    assert HK.hausdorff(a, np.array([0.0, 1.0 + 1.0j, 3.0])) == abs(3.0 - (1.0 + 1.0j))
    assert HK.hausdorff(np.array([0.0]), np.array([0.5])) == 0.5


def test_rng_counts_against_printed_shares():
    vals = {}
    with open(os.path.join(GOLDEN, "era_rng_percentages.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    m, n, s = int(vals["m"]), int(vals["n"]), int(vals["s"])
    ell_r = int(vals["r"] + vals["rho"])
    ell_l = int(math.ceil(1.5 * ell_r))
    krp = HK.rng_count_block(m, n, s, s, ell_r, ell_l)
    gauss = HK.rng_count_block_gauss(m, n, s, s, ell_r, ell_l)
    randera = n * s * ell_r
    assert math.floor(1000 * krp / randera) / 10 == vals["pct_of_randera"]
    assert math.floor(1000 * krp / gauss) / 10 == vals["pct_of_rgauss"]
    # the oracle's actual draws have exactly that many entries
    o1, o2, p1, p2 = HK.sketch_factors(0, s, m, n, 3, 4)
    assert o1.size + o2.size + p1.size + p2.size == HK.rng_count_block(m, n, s, s, 3, 4)


# ---- Nystrom approximation (the remark after Alg. 6) and its eigensolver ----

@pytest.mark.parametrize("n", [1, 2, 7, 20])
def test_jacobi_eig_matches_lapack(n):
    """Two-sided Jacobi against LAPACK's symmetric eigensolver, on an
    indefinite matrix: eigenvalues, A V = V diag(w), V orthogonal."""
    from oracle import linalg as LA
    rng = np.random.default_rng(40 + n)
    a = rng.standard_normal((n, n))
    a = a + a.T
    w, v = LA.jacobi_eig(a)
    scale = np.linalg.norm(a)
    assert np.all(np.diff(w) <= 0)
    assert np.allclose(w, np.sort(np.linalg.eigvalsh(a))[::-1], atol=1e-12 * scale)
    assert np.linalg.norm(a @ v - v * w) <= 1e-12 * scale
    assert np.linalg.norm(v.T @ v - np.eye(n)) <= 1e-12


def _spsd_spec(order, m, s, seed=11):
    return HankelSpec("nys", order, m, m, s, 0.9, seed, r=order, ell_r=order, ell_l=order)


def test_symmetric_system_is_spsd():
    """The generator's block Hankel matrix is symmetric PSD of rank <= order."""
    from synth import symmetric_markov_parameters
    h = HK.block_hankel(symmetric_markov_parameters(_spsd_spec(6, 3, 10)))
    assert np.linalg.norm(h - h.T) <= 1e-13 * np.linalg.norm(h)
    w = np.linalg.eigvalsh(h)
    assert w.min() >= -1e-12 * w.max()
    assert np.sum(w > 1e-10 * w.max()) <= 6


@pytest.mark.parametrize("order,m,s,ell", [(6, 3, 10, 10), (4, 2, 9, 4)])
def test_nystrom_exact_for_low_rank(order, m, s, ell):
    """rank(M) <= l: the column space of M Omega is that of M, and M_nys = M;
    its eigenpairs are M's (LAPACK), U orthonormal."""
    from synth import symmetric_markov_parameters
    blocks = symmetric_markov_parameters(_spsd_spec(order, m, s))
    out = HK.nystrom(blocks, order, ell, seed=3)
    h = out["H"]
    assert out["kept"] == order
    assert np.linalg.norm(out["M"] - h) <= 1e-9 * np.linalg.norm(h)
    w = np.sort(np.linalg.eigvalsh(h))[::-1][:order]
    assert np.allclose(out["L"], w, rtol=0, atol=1e-9 * w[0])
    u = out["U"]
    assert np.linalg.norm(u.T @ u - np.eye(order)) <= 1e-10
    assert np.linalg.norm(u * out["L"] @ u.T - h) <= 1e-9 * np.linalg.norm(h)


def test_nystrom_below_m_and_eckart_young():
    """l < rank(M): M - M_nys is PSD (M_nys = M^{1/2} P M^{1/2} with P an
    orthogonal projector), M_nys is PSD of rank <= l, and its error is at
    least the best rank-l error sqrt(sum_{i > l} lambda_i^2)."""
    from synth import symmetric_markov_parameters
    blocks = symmetric_markov_parameters(_spsd_spec(12, 4, 16))
    ell = 7
    out = HK.nystrom(blocks, 5, ell, seed=9)
    h, mn = out["H"], out["M"]
    nh = np.linalg.norm(h)
    assert np.linalg.eigvalsh(h - mn).min() >= -1e-10 * nh
    wn = np.linalg.eigvalsh(mn)
    assert wn.min() >= -1e-10 * nh
    assert np.sum(wn > 1e-10 * nh) <= ell
    lam = np.sort(np.linalg.eigvalsh(h))[::-1]
    assert np.linalg.norm(h - mn) >= np.sqrt(np.sum(lam[ell:] ** 2)) * (1 - 1e-12)
    # the top r eigenpairs returned are those of M_nys
    wtop = np.sort(wn)[::-1][:5]
    assert np.allclose(out["L"], wtop, rtol=0, atol=1e-10 * nh)


def test_nystrom_core_from_structured_sketch():
    """Omega^T M Omega from the structured sketch of Eq. (4.1) (what the CUDA
    path forms) equals the oracle's explicit C."""
    from synth import symmetric_markov_parameters
    blocks = symmetric_markov_parameters(_spsd_spec(6, 3, 10))
    out = HK.nystrom(blocks, 4, 8, seed=21)
    s = (blocks.shape[2] + 1) // 2
    o1, o2, _, _ = HK.sketch_factors(21, s, 3, 3, 8, 1)
    y = HK.structured_sketch(blocks, o1, o2)
    c = T.khatri_rao(o1, o2).T @ y
    assert np.linalg.norm(0.5 * (c + c.T) - out["C"]) <= 1e-12 * np.linalg.norm(c)


# ---- two-level block Hankel matrices (Sec. 4.3) ----

def test_block_hankel2_is_the_kronecker_sum():
    """M = sum_{k1,k2} E_{k1} kron E_{k2} kron H_{k1,k2} with the 0/1 patterns
    of Sec. 4.2 at both levels, from explicit Kronecker products."""
    from synth import two_level_markov_parameters
    b = two_level_markov_parameters(3, 2, 3, 4, 3, seed=1)
    m, n = 2, 3
    s1, s2 = 4, 3
    ref = 0.0
    for k1 in range(1, 2 * s1):
        for k2 in range(1, 2 * s2):
            ref = ref + np.kron(HK.hankel_pattern(s1, k1),
                                np.kron(HK.hankel_pattern(s2, k2), b[:, :, k1 - 1, k2 - 1]))
    assert np.array_equal(HK.block_hankel2(b), ref)


def test_structured_sketch2_identity():
    """Two-level Eq. (4.1): M (O1 kr O2 kr O3) and M^T (P1 kr P2 kr P3)."""
    from synth import two_level_markov_parameters
    b = two_level_markov_parameters(4, 3, 2, 5, 4, seed=2)
    h = HK.block_hankel2(b)
    rng = np.random.default_rng(3)
    om = [rng.standard_normal((r, 6)) for r in (5, 4, 2)]
    ps = [rng.standard_normal((r, 7)) for r in (5, 4, 3)]
    y = HK.structured_sketch2(b, *om)
    z = HK.structured_sketch2(b, *ps, transpose=True)
    assert np.linalg.norm(y - h @ T.khatri_rao_list(om)) <= 1e-12 * np.linalg.norm(y)
    assert np.linalg.norm(z - h.T @ T.khatri_rao_list(ps)) <= 1e-12 * np.linalg.norm(z)


def test_single_pass_svd2_exact_for_low_rank():
    """rank(M) <= order <= l_r: the two-sided single-pass approximation
    reproduces M, and its singular values are LAPACK's."""
    from synth import two_level_markov_parameters
    order = 5
    b = two_level_markov_parameters(order, 3, 2, 6, 5, seed=4)
    out = HK.single_pass_svd2(b, order, order + 4, 2 * (order + 4), seed=5)
    h = out["H"]
    assert np.linalg.matrix_rank(h, tol=1e-10 * np.linalg.norm(h)) <= order
    approx = (out["U"] * out["S"]) @ out["V"].T
    assert np.linalg.norm(approx - h) <= 1e-9 * np.linalg.norm(h)
    sv = np.linalg.svd(h, compute_uv=False)[:order]
    assert np.allclose(out["S"], sv, rtol=0, atol=1e-9 * sv[0])
