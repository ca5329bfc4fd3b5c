"""krp_qr_noalloc: the thin QR for callers that may not allocate device memory.

It must give the same Q and R as krp_qr (which may grow its workspace with
cudaMalloc) on the same input, call after call, using only the library's fixed
scratch array.  Kept in its own file, collected last, so that a failure here
never hides the results of the other GPU tests.
"""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, mat_to_dev, mat_from_dev, empty_mat
from oracle import philox

pytestmark = pytest.mark.gpu


def _qr_reference(ctx, yd, m, l):
    import torch
    import paper_2507_23207_gb300 as K
    q = empty_mat(m, l, torch.float64)
    r = empty_mat(l, l, torch.float64)
    K.krp_qr(ctx, [yd], [m], [l], [q], [r])
    return q, r


def test_noalloc_qr_matches_krp_qr_on_consecutive_calls():
    torch = require_gpu()
    import paper_2507_23207_gb300 as K
    lib = K.load_library()
    ctx = K.Context(0)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(17)
    shapes = [(1024, 48), (200, 30), (1024, 48)]  # the third call repeats the first shape
    for call, (m, l) in enumerate(shapes):
        y = philox.round_to_f32(rng.standard_normal((m, l)))
        yd = mat_to_dev(y, torch.float32)
        q = empty_mat(m, l, torch.float64)
        r = empty_mat(l, l, torch.float64)
        st = lib.krp_qr_noalloc(yd.data_ptr(), m, l, q.data_ptr(), r.data_ptr(), stream)
        assert st == K.KRP_OK, (call, st)
        qr_, rr_ = _qr_reference(ctx, yd, m, l)
        torch.cuda.synchronize()
        qg, rg = mat_from_dev(q, m, l), mat_from_dev(r, l, l)
        np.testing.assert_allclose(qg, mat_from_dev(qr_, m, l), atol=1e-12)
        np.testing.assert_allclose(rg, mat_from_dev(rr_, l, l), atol=1e-12 * np.linalg.norm(y))
        assert np.linalg.norm(qg.T @ qg - np.eye(l)) <= 1e-13
        np.testing.assert_allclose(qg @ rg, y, atol=1e-12 * np.linalg.norm(y))
    ctx.close()


def test_noalloc_qr_allocates_nothing_and_handles_no_r_and_rank_deficiency():
    """After a first call (which may load the library's device code), further
    calls leave the device's free memory unchanged; R may be NULL; a Y with a
    zero column and a repeated column (rank-deficient: collapsed pivots are
    refilled through the scratch's mask) still gives an orthonormal Q whose
    range holds Y, and the same Q as krp_qr (R is compared on full-rank input
    above: where a pivot collapses, its entries are set by FP64 sums whose
    order is not fixed, so only Q and the projection are unique here)."""
    torch = require_gpu()
    import paper_2507_23207_gb300 as K
    lib = K.load_library()
    ctx = K.Context(0)
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(23)
    m, l = 700, 24
    y = philox.round_to_f32(rng.standard_normal((m, l)))
    y[:, 5] = 0.0
    y[:, 9] = y[:, 2]
    yd = mat_to_dev(y, torch.float32)
    q = empty_mat(m, l, torch.float64)
    r = empty_mat(l, l, torch.float64)
    assert lib.krp_qr_noalloc(yd.data_ptr(), m, l, q.data_ptr(), r.data_ptr(), stream) == K.KRP_OK
    qr_, rr_ = _qr_reference(ctx, yd, m, l)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert lib.krp_qr_noalloc(yd.data_ptr(), m, l, q.data_ptr(), None, stream) == K.KRP_OK
        assert lib.krp_qr_noalloc(yd.data_ptr(), m, l, q.data_ptr(), r.data_ptr(),
                                  stream) == K.KRP_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    qg, rg = mat_from_dev(q, m, l), mat_from_dev(r, l, l)
    assert np.all(np.isfinite(qg))
    assert np.linalg.norm(qg.T @ qg - np.eye(l)) <= 1e-12
    assert np.linalg.norm(y - qg @ (qg.T @ y)) <= 1e-12 * np.linalg.norm(y)
    np.testing.assert_allclose(qg, mat_from_dev(qr_, m, l), atol=1e-10)
    assert np.all(np.isfinite(rg))
    ctx.close()


def test_noalloc_qr_rejects_requests_beyond_its_scratch():
    torch = require_gpu()
    import paper_2507_23207_gb300 as K
    lib = K.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    small = empty_mat(8, 4, torch.float32)
    out = empty_mat(8, 4, torch.float64)
    # m*l + 4 l^2 + 2 doubles must fit the 4 MiB scratch
    m, l = 16384, 48
    assert m * l + 4 * l * l + 2 > K.KRP_QR_NOALLOC_MAX_DOUBLES
    assert lib.krp_qr_noalloc(small.data_ptr(), m, l, out.data_ptr(), None, stream) == K.KRP_EINVAL
    assert lib.krp_qr_noalloc(small.data_ptr(), 100, 65, out.data_ptr(), None, stream) == K.KRP_EINVAL
    assert lib.krp_qr_noalloc(small.data_ptr(), 3, 4, out.data_ptr(), None, stream) == K.KRP_EINVAL
    assert lib.krp_qr_noalloc(None, 8, 4, out.data_ptr(), None, stream) == K.KRP_EINVAL
