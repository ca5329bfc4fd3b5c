"""Pins of the oracle's sensor placement (Sec. 6).

* The pivots equal LAPACK's column-pivoted QR (scipy, geqp3) on inputs whose
  pivot decisions have a clear margin.
* Interpolation: P^T A = I, i.e. A[idx, :] is the identity.
* Exactness: a tensor in the span of the factors (T = C x {Q_i}) is recovered
  exactly from its values on the sensor grid.
* The selected rows are a usable basis: ||(P^T Q)^{-1}||_2 stays within
  sqrt(N l) 2^l, the worst-case growth bound of the greedy pivoted-QR
  selection (the DEIM error constant).
* l = N: every index is selected once (the order is not unique).
"""

import numpy as np
import pytest

from oracle import sensor as SE
from oracle import tucker as TK
from synth import haar


@pytest.mark.parametrize("n,ell,seed", [(40, 5, 1), (150, 12, 2), (90, 10, 3)])
def test_pivots_match_lapack(n, ell, seed):
    import scipy.linalg as sl
    q = haar(n, ell, np.random.default_rng(seed))
    assert SE.pivot_margins(q).min() > 1e-9
    idx = SE.pivoted_qr_select(q)
    _, _, piv = sl.qr(q.T, pivoting=True, mode="economic")
    assert np.array_equal(idx, piv[:ell])
    assert len(set(idx.tolist())) == ell


def test_square_factor_selects_every_index():
    """l = N: all column norms of Q^T are 1 (ties at every step), so the order
    is not unique but the set is: every index once."""
    q = haar(8, 8, np.random.default_rng(4))
    idx = SE.pivoted_qr_select(q)
    assert sorted(idx.tolist()) == list(range(8))
    a = SE.interpolation_factor(q, idx)
    assert np.linalg.norm(a[idx, :] - np.eye(8)) <= 1e-12


@pytest.mark.parametrize("n,ell,seed", [(40, 5, 5), (150, 12, 6)])
def test_interpolation_factor_is_identity_on_sensors(n, ell, seed):
    q = haar(n, ell, np.random.default_rng(seed))
    idx = SE.pivoted_qr_select(q)
    a = SE.interpolation_factor(q, idx)
    assert np.linalg.norm(a[idx, :] - np.eye(ell)) <= 1e-12
    # A spans the same space as Q
    assert np.linalg.norm(a - q @ (q.T @ a)) <= 1e-12 * np.linalg.norm(a)
    # DEIM error constant ||(P^T Q)^{-1}||_2 stays moderate for the greedy pick
    assert np.linalg.norm(np.linalg.inv(q[idx, :]), 2) <= np.sqrt(n * ell) * 2.0 ** ell


def test_exact_recovery_in_the_span():
    rng = np.random.default_rng(9)
    dims, ells = (30, 24, 18), (5, 4, 3)
    qs = [haar(n, l, rng) for n, l in zip(dims, ells)]
    core = rng.standard_normal(ells)
    t = TK.reconstruct(core, qs)
    idxs = [SE.pivoted_qr_select(q) for q in qs]
    a = [SE.interpolation_factor(q, i) for q, i in zip(qs, idxs)]
    t_hat = t[np.ix_(*idxs)]
    out = SE.sensor_reconstruct(t_hat, a)
    assert np.linalg.norm(out - t) <= 1e-12 * np.linalg.norm(t)
