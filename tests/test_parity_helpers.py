"""CPU checks of the comparison helpers in tests/parity.py."""

import math

import numpy as np
import pytest

from oracle import tucker as TK
from tests.parity import (U_F32, check_error_value, eval_bound, projector_distance,
                          recon_distance)


def _orth(rng, n, r):
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


@pytest.mark.parametrize("dims,ranks", [((9, 8, 7), (3, 2, 4)), ((6, 5, 4, 3), (2, 2, 2, 2))])
def test_recon_distance_equals_explicit(dims, ranks):
    rng = np.random.default_rng(3)
    g1 = rng.standard_normal(ranks)
    q1 = [_orth(rng, n, r) for n, r in zip(dims, ranks)]
    # a nearby second approximation: perturbed core, rotated and perturbed factors
    g2 = g1 + 1e-3 * rng.standard_normal(ranks)
    q2 = [_orth(rng, r, r) for r in ranks]
    q2 = [np.linalg.qr(q @ o + 1e-4 * rng.standard_normal(q.shape))[0] for q, o in zip(q1, q2)]
    explicit = np.linalg.norm(TK.reconstruct(g1, q1) - TK.reconstruct(g2, q2))
    assert recon_distance(g1, q1, g2, q2) == pytest.approx(explicit, rel=1e-10)
    # same approximation in another basis: distance 0
    rot = [_orth(rng, r, r) for r in ranks]
    g1r = g1
    for i, o in enumerate(rot):
        g1r = np.moveaxis(np.tensordot(o.T, g1r, axes=(1, i)), 0, i)
    q1r = [q @ o for q, o in zip(q1, rot)]
    assert recon_distance(g1, q1, g1r, q1r) <= 1e-12 * np.linalg.norm(g1)


def test_projector_distance_equals_explicit():
    rng = np.random.default_rng(4)
    qa = _orth(rng, 30, 5)
    qb = np.linalg.qr(qa + 1e-3 * rng.standard_normal(qa.shape))[0]
    explicit = np.linalg.norm(qa @ qa.T - qb @ qb.T) / math.sqrt(5)
    assert projector_distance(qa, qb) == pytest.approx(explicit, rel=1e-8)
    assert projector_distance(qa, qa @ _orth(rng, 5, 5)) <= 1e-14


def test_error_value_check_rejects_wrong_residuals():
    """At the 64^3 workload's error level (e ~ 2.3e-6, l = 5 per mode) a
    residual of 0 or of 1e-5 fails, a value within the rounding bound passes."""
    e = 2.3e-6
    rho = eval_bound((5, 5, 5), (64, 64, 64), 1.0, e)
    assert rho < 0.2 * e
    eta = 3e-8
    check_error_value(e * (1 + 1e-3), e, e, eta, rho)
    for wrong in (0.0, 1e-5):
        with pytest.raises(AssertionError):
            check_error_value(wrong, e, e, eta, rho)
    # at the 1024^3 workload (l = 32, e ~ 1e-4) rho is below 1e-3 e
    assert eval_bound((32, 32, 32), (1024,) * 3, 1.0, 1e-4) < 1e-7
    assert U_F32 == 2.0 ** -24
