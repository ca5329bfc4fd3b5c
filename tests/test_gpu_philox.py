"""a1 parity: the device Philox stream and Gaussian factors against the oracle.

The uint32 words must be bit-exact.  The Gaussian values go through FP64
log/sincospi on the device and log/cos/sin in numpy, so FP64 factors agree to
a few ulp and FP32/BF16 factors agree exactly except where the FP64 values
straddle a rounding boundary (then by one ulp of the narrow type).
"""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, mat_from_dev, empty_mat
from oracle import philox

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("seed,c1,c2,c3,first,n", [
    (0, 0, 0, 0, 0, 1000),
    (12345, 2, 7, 0, 2**32 - 10, 20),  # counter wraps its 32-bit word
    (2**63 + 5, 1, 65, 1, 77, 513),
    (2**64 - 1, 3, 0, 2, 123456789, 4096),
])
def test_philox_words_bit_exact(ctx, seed, c1, c2, c3, first, n):
    import torch
    import paper_2507_23207_gb300 as K
    out = torch.zeros(4 * n, dtype=torch.int32, device=dev())
    K.krp_philox_words(ctx, seed, c1, c2, c3, first, n, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    blk = (np.arange(n, dtype=np.uint64) + np.uint64(first)) & np.uint64(0xFFFFFFFF)
    ref = np.stack(philox.philox4x32_10(blk, c1, c2, c3, seed & 0xFFFFFFFF, seed >> 32), axis=1)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("rows,ell", [(64, 10), (1024, 48), (7, 3), (1, 1), (200, 30), (33, 5)])
def test_gaussian_factors_f64(ctx, rows, ell):
    import torch
    import paper_2507_23207_gb300 as K
    rows_l = [rows, rows + 3, max(1, rows - 1)]
    ts = [empty_mat(r, ell, torch.float64) for r in rows_l]
    K.krp_gen_factors(ctx, 99, 5, 0, rows_l, ell, ts)
    torch.cuda.synchronize()
    for j, (r, t) in enumerate(zip(rows_l, ts)):
        ref = philox.gaussian_factor(99, j, 5, 0, r, ell)
        np.testing.assert_allclose(mat_from_dev(t, r, ell), ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("dtype_name", ["float32", "bfloat16"])
def test_gaussian_factors_narrow_types(ctx, dtype_name):
    import torch
    import paper_2507_23207_gb300 as K
    dt = getattr(torch, dtype_name)
    rows, ell = 1024, 48
    ts = [empty_mat(rows, ell, dt), None, empty_mat(37, ell, dt)]
    K.krp_gen_factors(ctx, 7, 0, 1, [rows, 5, 37], ell, ts)
    torch.cuda.synchronize()
    rnd = philox.round_to_f32 if dtype_name == "float32" else philox.round_to_bf16
    for j, r in [(0, rows), (2, 37)]:
        ref = rnd(philox.gaussian_factor(7, j, 0, 1, r, ell))
        got = mat_from_dev(ts[j], r, ell)
        diff = got != ref
        assert diff.mean() < 1e-3
        ulp = 2.0 ** -23 if dtype_name == "float32" else 2.0 ** -7
        assert np.all(np.abs(got - ref) <= ulp * np.maximum(np.abs(ref), 2.0 ** -100) * 1.0001)


def test_prefix_consistent_columns(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    a = empty_mat(50, 9, torch.float32)
    b = empty_mat(50, 4, torch.float32)
    K.krp_gen_factors(ctx, 3, 2, 0, [50], 9, [a])
    K.krp_gen_factors(ctx, 3, 2, 0, [50], 4, [b])
    torch.cuda.synchronize()
    assert np.array_equal(mat_from_dev(a, 50, 9)[:, :4], mat_from_dev(b, 50, 4))


def test_invalid_arguments(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    t = empty_mat(4, 4, torch.float32)
    with pytest.raises(K.KrpError) as e:
        K.krp_gen_factors(ctx, 0, 0, 0, [4], 0, [t])
    assert e.value.status == K.KRP_EINVAL
    with pytest.raises(K.KrpError):
        K.krp_gen_factors(ctx, 0, 0, 0, [0], 4, [t])
