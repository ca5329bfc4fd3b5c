"""Pins of the oracle's FP8 E4M3 per-slab quantiser (oracle/quant.py).

* The code table, decoded by the format's formula, against torch's
  float8_e4m3fn (an independent implementation of the OCP E4M3 format).
* The rounding (RN-even) against torch's FP32 -> float8_e4m3fn conversion,
  code for code, on random values, exact ties and subnormals; saturation of
  finite overflow by its definition.
* The rounding error bounds of a 3-bit mantissa: half an ulp, i.e. 2^-4
  relative in the normal range and 2^-10 absolute among subnormals.
* Per-slab scaling: the largest entry of each slab lands on +-448, the
  stored copy is within those bounds of the FP32 tensor slab by slab, and
  the scale of a slab does not depend on the other slabs.
"""

import numpy as np
import pytest

from oracle import quant


def _torch_codes(values32):
    import torch
    t = torch.from_numpy(np.asarray(values32, dtype=np.float32))
    return t.to(torch.float8_e4m3fn).view(torch.uint8).numpy()


def test_code_table_matches_torch_float8_e4m3fn():
    import torch
    codes = np.arange(256)
    mine = quant.e4m3_decode(codes)
    ref = torch.from_numpy(codes.astype(np.uint8)).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(np.isnan(mine), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.array_equal(mine[ok], ref[ok])
    # format constants from the formula
    assert np.nanmax(mine) == quant.E4M3_MAX == 2.0 ** 8 * (1 + 6 / 8)
    assert mine[1] == quant.E4M3_MIN_SUBNORMAL
    assert mine[8] == quant.E4M3_MIN_NORMAL
    # positive codes are strictly increasing up to 0x7E
    assert np.all(np.diff(mine[:0x7F]) > 0)


def test_rounding_matches_torch_conversion_code_for_code():
    rng = np.random.default_rng(5)
    mags = 2.0 ** rng.uniform(-12, np.log2(440), 20000)
    x = (mags * rng.choice([-1.0, 1.0], mags.size)).astype(np.float32)
    grid = quant.e4m3_decode(np.arange(0x7F))
    mids = ((grid[:-1] + grid[1:]) / 2).astype(np.float32)   # exact ties (representable in FP32)
    specials = np.array([0.0, -0.0, 448.0, -448.0, 449.0, 464.0, 2.0 ** -10, 2.0 ** -9,
                         1.5 * 2.0 ** -10, 17.0, 19.0, 3.0e-39], dtype=np.float32)
    allx = np.concatenate([x, mids, -mids, specials])
    assert np.array_equal(quant.round_to_e4m3_codes(allx), _torch_codes(allx))


def test_saturation_and_nan():
    big = np.array([448.0, 480.0, 1.0e4, 3.0e38, np.inf, -1.0e4, -np.inf])
    assert np.array_equal(quant.round_to_e4m3(big),
                          np.array([448.0, 448.0, 448.0, 448.0, 448.0, -448.0, -448.0]))
    assert np.isnan(quant.round_to_e4m3(np.array([np.nan])))[0]


def test_rounding_error_is_half_an_ulp():
    rng = np.random.default_rng(6)
    v = (2.0 ** rng.uniform(-14, np.log2(448), 50000)).astype(np.float32).astype(np.float64)
    q = quant.round_to_e4m3(v)
    err = np.abs(q - v)
    normal = v >= quant.E4M3_MIN_NORMAL
    assert np.all(err[normal] <= 2.0 ** -4 * v[normal])
    assert np.all(err[~normal] <= 2.0 ** -10)
    # and it is the nearest grid value: no grid point is strictly closer
    grid = quant.e4m3_decode(np.arange(0x7F))
    best = np.min(np.abs(grid[None, :] - v[:2000, None]), axis=1)
    assert np.array_equal(err[:2000], best)


def test_slab_scales_put_each_slab_maximum_on_448():
    rng = np.random.default_rng(7)
    # slabs of very different magnitudes, one all-zero slab
    x = rng.standard_normal((9, 7, 6)) * (10.0 ** np.arange(-3, 3))[None, None, :]
    x[:, :, 2] = 0.0
    codes, s = quant.quantize_slabs(x)
    q = quant.e4m3_decode(codes)
    for t in range(x.shape[-1]):
        if t == 2:
            assert s[t] == 1.0 and np.all(q[..., t] == 0)
            continue
        assert np.max(np.abs(q[..., t])) == 448.0
        amax = np.max(np.abs(x[..., t].astype(np.float32)))
        assert s[t] == np.float32(amax / np.float32(448.0))
    # the scale of a slab depends on that slab only
    x2 = x.copy()
    x2[..., 0] *= 1000.0
    _, s2 = quant.quantize_slabs(x2)
    assert np.array_equal(s2[1:], s[1:])


def test_dequantized_slabs_within_the_rounding_bound():
    rng = np.random.default_rng(8)
    x = rng.standard_normal((16, 12, 10)) * rng.uniform(0.01, 100.0, 10)[None, None, :]
    codes, s = quant.quantize_slabs(x)
    xt = quant.dequantize_slabs(codes, s)
    x32 = x.astype(np.float32).astype(np.float64)
    # q = E4M3(fl32(x/s)): the FP32 quotient adds 2^-24 relative before the
    # E4M3 rounding; subnormal codes add at most 2^-10 s absolute
    bound = (2.0 ** -4 + 2.0 ** -23) * np.abs(x32) + 2.0 ** -10 * s[None, None, :]
    assert np.all(np.abs(xt - x32) <= bound)
    rel = np.linalg.norm(xt - x32) / np.linalg.norm(x32)
    assert rel <= 2.0 ** -4
    # the stored values are exact products q * s (no rounding in FP64)
    q = quant.e4m3_decode(codes)
    assert np.array_equal(xt / s[None, None, :], q)


@pytest.mark.parametrize("shape", [(5,), (3, 4), (2, 3, 4, 5)])
def test_quantize_any_order(shape):
    rng = np.random.default_rng(9)
    x = rng.standard_normal(shape)
    codes, s = quant.quantize_slabs(x)
    assert codes.shape == x.shape and codes.dtype == np.uint8
    assert s.shape == (shape[-1],)


def test_fp8_storage_fails_the_accuracy_criterion_on_a_decaying_core():
    """E4M3 with per-slab scales leaves relative noise of ~2.6e-2 in X (BF16:
    ~1.7e-3).  On a decaying core (0.8^(i+j+k), 120^3, rank 20 from l = 30,
    approximation error ~1.2e-2) that noise dominates the sketch: the error
    is several times the FP32 form's whether X is FP8 throughout or only in
    the sketch (the core then taken from the FP32 data), because the range
    finder spends its extra columns on the quantisation noise.  A 1.05x
    criterion therefore rules FP8 storage out for such tensors; BF16 (1.18x)
    is the closest of the short formats."""
    from oracle import philox
    from oracle import tucker as TK
    from oracle.tensor import multi_ttm
    from synth.tucker import TuckerSpec, tucker_tensor
    spec = TuckerSpec("q8", (120, 120, 120), (40, 40, 40), 0.0, 0.8, 1003, (20, 20, 20),
                      (30, 30, 30))
    x, _, _ = tucker_tensor(spec)
    x32 = philox.round_to_f32(x)
    codes, s = quant.quantize_slabs(x32)
    x8 = quant.dequantize_slabs(codes, s)
    noise = np.linalg.norm(x8 - x32) / np.linalg.norm(x32)
    assert 1.0e-2 < noise < 2.0 ** -4

    def err(x_sketch, x_core):
        o = TK.rhosvd_krp(x_sketch, [30] * 3, 0, memo=True, omega_round="f32")
        g = multi_ttm(x_core, [q.T for q in o["Q"]])
        g2, q2 = TK.truncate_core(g, o["Q"], [20] * 3)
        return TK.rel_error(x, g2, q2)

    e32 = err(x32, x32)
    assert err(x8, x8) > 3.0 * e32
    assert err(x8, x32) > 3.0 * e32
