"""a4/a5 parity: FP64 Householder QR and the multi-TTM core against the oracle."""

import numpy as np
import pytest

from tests.gpu_util import (require_gpu, dev, mat_to_dev, mat_from_dev, empty_mat,
                            tensor_to_dev, tensor_from_dev, rel)
from oracle import linalg as L, philox, tensor as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("m,l", [(64, 10), (1024, 48), (200, 30), (33, 33), (1000, 1), (129, 64)])
def test_qr_matches_oracle(ctx, m, l):
    import torch
    import paper_2507_23207_gb300 as K
    y = philox.round_to_f32(np.random.default_rng(m + l).standard_normal((m, l)))
    yd = mat_to_dev(y, torch.float32)
    q = empty_mat(m, l, torch.float64)
    r = empty_mat(l, l, torch.float64)
    K.krp_qr(ctx, [yd], [m], [l], [q], [r])
    torch.cuda.synchronize()
    qo, ro = L.householder_qr(y)
    qg, rg = mat_from_dev(q, m, l), mat_from_dev(r, l, l)
    assert np.linalg.norm(qg.T @ qg - np.eye(l)) <= 1e-13
    np.testing.assert_allclose(qg, qo, atol=1e-12)
    np.testing.assert_allclose(rg, ro, atol=1e-12 * np.linalg.norm(y))
    assert np.all(np.diag(rg) >= 0)


def test_qr_batched_and_rank_deficient(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    rng = np.random.default_rng(3)
    shapes = [(50, 9), (300, 20), (17, 17)]
    ys = []
    for m, l in shapes:
        a = rng.standard_normal((m, 4)) @ rng.standard_normal((4, l))
        a[:, l // 2] = 0.0
        ys.append(philox.round_to_f32(a))
    yd = [mat_to_dev(y, torch.float32) for y in ys]
    qs = [empty_mat(m, l, torch.float64) for m, l in shapes]
    K.krp_qr(ctx, yd, [m for m, _ in shapes], [l for _, l in shapes], qs)
    torch.cuda.synchronize()
    for (m, l), y, q in zip(shapes, ys, qs):
        qg = mat_from_dev(q, m, l)
        assert np.linalg.norm(qg.T @ qg - np.eye(l)) <= 1e-13
        assert np.linalg.norm(y - qg @ (qg.T @ y)) <= 1e-12 * np.linalg.norm(y)


def test_qr_rejects_non_finite(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    y = np.ones((10, 3))
    y[4, 1] = np.nan
    yd = mat_to_dev(y, torch.float32)
    q = empty_mat(10, 3, torch.float64)
    with pytest.raises(K.KrpError) as e:
        K.krp_qr(ctx, [yd], [10], [3], [q])
    assert e.value.status == K.KRP_ENUMERIC
    with pytest.raises(K.KrpError) as e:
        K.krp_qr(ctx, [yd], [2], [3], [q])
    assert e.value.status == K.KRP_EINVAL


@pytest.mark.parametrize("dims,cols", [((37, 29, 23), (5, 4, 6)), ((16, 8, 4, 6), (3, 2, 4, 5)),
                                       ((130, 70, 33), (48, 20, 33)), ((64, 64, 64), (10, 10, 10))])
def test_multi_ttm_matches_oracle(ctx, dims, cols):
    import torch
    import paper_2507_23207_gb300 as K
    rng = np.random.default_rng(sum(dims))
    x = philox.round_to_f32(np.asfortranarray(rng.standard_normal(dims)))
    qs = [L.householder_qr(rng.standard_normal((n, c)))[0] for n, c in zip(dims, cols)]
    xd = tensor_to_dev(x, torch.float32)
    qd = [mat_to_dev(q, torch.float64) for q in qs]
    g = torch.empty(int(np.prod(cols)), dtype=torch.float32, device=dev())
    K.krp_multi_ttm(ctx, xd, dims, qd, cols, g)
    torch.cuda.synchronize()
    ref = T.multi_ttm(x, [q.T for q in qs])
    assert rel(tensor_from_dev(g, cols), ref) <= 1e-5
