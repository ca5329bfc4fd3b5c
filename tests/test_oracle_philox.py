"""Pins of the oracle's Philox4x32-10 stream and its Gaussian transform.

* Against an independent third-party implementation: Triton's Philox4x32
  (``triton.language.philox``), run by Triton's CPU interpreter in a
  subprocess, on the oracle's exact counter/key layout.
* Statistical: byte-level chi-square uniformity, Gaussian moments and a
  Kolmogorov-Smirnov test of the Box-Muller output.
* bfloat16 rounding against torch's CPU float32 -> bfloat16 conversion.
"""

import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from oracle import philox

TRITON_SCRIPT = textwrap.dedent("""
    import json, os, sys
    os.environ["TRITON_INTERPRET"] = "1"
    import numpy as np, torch, triton, triton.language as tl

    @triton.jit
    def kern(out_ptr, c0_ptr, c1, c2, c3, seed, N: tl.constexpr):
        offs = tl.arange(0, N)
        c0 = tl.load(c0_ptr + offs)
        z = c0 * 0
        a, b, c, d = tl.philox(seed, c0, z + c1, z + c2, z + c3, 10)
        tl.store(out_ptr + offs * 4 + 0, a)
        tl.store(out_ptr + offs * 4 + 1, b)
        tl.store(out_ptr + offs * 4 + 2, c)
        tl.store(out_ptr + offs * 4 + 3, d)

    cases = json.loads(sys.argv[1])
    res = []
    for (seed, c1, c2, c3, c0list) in cases:
        n = len(c0list)
        c0 = torch.tensor(c0list, dtype=torch.int64).to(torch.uint32)
        out = torch.zeros(4 * n, dtype=torch.uint32)
        kern[(1,)](out, c0, c1, c2, c3, seed, n)
        res.append([int(v) for v in out.tolist()])
    print(json.dumps(res))
""")


def _triton_available():
    try:
        import triton  # noqa: F401
        import triton.language as tl
        return hasattr(tl, "philox")
    except Exception:
        return False


@pytest.mark.skipif(not _triton_available(), reason="triton not installed")
def test_philox_matches_triton_reference_implementation(tmp_path):
    # counters: (block index c0, factor j, draw id, tag) with a 64-bit key
    cases = [
        [0, 0, 0, 0, list(range(16))],
        [12345, 2, 7, 0, [0, 1, 2, 1000, 65535, 2**31 + 5, 2**32 - 1, 77, 3, 9,
                          123456, 42, 8, 16, 31, 4095]],
        [2**40 + 99, 1, 0, 1, [5 * i + 3 for i in range(16)]],
        [2**64 - 1, 3, 65, 2, [2**32 - 1 - i for i in range(16)]],
    ]
    script = tmp_path / "tri.py"
    script.write_text(TRITON_SCRIPT)
    env = dict(os.environ)
    env["TRITON_INTERPRET"] = "1"
    out = subprocess.run([sys.executable, str(script), json.dumps(cases)],
                         capture_output=True, text=True, env=env, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    ref = json.loads(out.stdout.strip().splitlines()[-1])
    for (seed, c1, c2, c3, c0list), words in zip(cases, ref):
        w = philox.philox4x32_10(np.array(c0list, dtype=np.uint64), c1, c2, c3,
                                 seed & 0xFFFFFFFF, seed >> 32)
        mine = np.stack(w, axis=1).reshape(-1).astype(np.int64)
        assert np.array_equal(mine, np.array(words, dtype=np.int64)), (seed, c1)


def test_philox_words_uniform_bytes_chi_square():
    from scipy import stats
    w = philox.factor_words(seed=2024, factor=0, draw=0, tag=0, rows=4096, cols=64)
    b = w.reshape(-1).view(np.uint8)
    counts = np.bincount(b, minlength=256)
    chi2 = np.sum((counts - b.size / 256) ** 2 / (b.size / 256))
    p = stats.chi2.sf(chi2, df=255)
    assert p > 1e-4, p


def test_philox_streams_differ_by_counter_fields():
    base = philox.factor_words(7, 0, 0, 0, 64, 4)
    for args in [(7, 1, 0, 0), (7, 0, 1, 0), (7, 0, 0, 1), (8, 0, 0, 0)]:
        other = philox.factor_words(*args, 64, 4)
        # a changed counter/key field changes (essentially) every word
        assert np.mean(base == other) < 0.01


def test_gaussian_moments_and_ks():
    from scipy import stats
    z = philox.gaussian_factor(seed=99, factor=1, draw=3, tag=0, rows=1000, cols=200)
    x = z.reshape(-1)
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    kurt = np.mean(x ** 4) / np.mean(x ** 2) ** 2
    assert abs(kurt - 3.0) < 5 * np.sqrt(24.0 / n)
    assert stats.kstest(x, "norm").pvalue > 1e-4


def test_gaussian_layout_column_major_lanes():
    rows, cols = 7, 5
    z = philox.gaussian_factor(3, 2, 1, 0, rows, cols)
    w = philox.factor_words(3, 2, 1, 0, rows, cols)
    for e in [0, 1, 2, 3, 4, 13, 34]:
        i, k = e % rows, e // rows
        blk, lane = divmod(e, 4)
        wa, wb = (w[blk, 0], w[blk, 1]) if lane < 2 else (w[blk, 2], w[blk, 3])
        ua = (float(wa) + 0.5) / 2 ** 32
        ub = (float(wb) + 0.5) / 2 ** 32
        rho = np.sqrt(-2 * np.log(ua))
        ref = rho * (np.cos(2 * np.pi * ub) if lane % 2 == 0 else np.sin(2 * np.pi * ub))
        assert z[i, k] == pytest.approx(ref, rel=1e-15, abs=1e-15)


def test_prefix_consistency_of_columns():
    # the first l' columns of an l-column factor do not depend on l
    a = philox.gaussian_factor(5, 0, 0, 0, 33, 10)
    b = philox.gaussian_factor(5, 0, 0, 0, 33, 4)
    assert np.array_equal(a[:, :4], b)


def test_bf16_rounding_matches_torch():
    import torch
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        np.array([1.0, -1.0, 0.0, 1.00390625, 1.01171875, 3.0e-39])])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(philox.round_to_bf16(x), ref)


def test_krp_columns_are_isotropic():
    """Sec. 2.5: a column of Omega_1 kr Omega_2 (independent standard Gaussian
    factors) has E[w w^T] = I.  Monte Carlo over 20000 columns drawn from the
    Philox stream at n = (3, 4).  The tolerance is 5 sigma of the sample
    mean: an entry of w w^T is a product of four standard normal factors,
    with variance at most E[x^4] E[y^4] - 1 = 8 (diagonal) and at most 3
    (off-diagonal).  A stream that repeated columns or correlated the two
    factors would fail it."""
    cols = 20000
    o1 = philox.gaussian_factor(11, 0, 0, philox.TAG_OMEGA, 3, cols)
    o2 = philox.gaussian_factor(11, 1, 0, philox.TAG_OMEGA, 4, cols)
    # column k of the Khatri-Rao product: kron(o1[:, k], o2[:, k])
    w = (o1[:, None, :] * o2[None, :, :]).reshape(12, cols)
    cov = w @ w.T / cols
    diag = np.diag(cov)
    off = cov - np.diag(diag)
    assert np.max(np.abs(diag - 1.0)) <= 5 * np.sqrt(8.0 / cols)
    assert np.max(np.abs(off)) <= 5 * np.sqrt(3.0 / cols)
    # the two factors of one column are independent draws (different counters)
    assert abs(np.corrcoef(o1[0], o2[0])[0, 1]) <= 5 / np.sqrt(cols)


def test_key_schedule_constants_from_their_closed_forms():
    """Salmon et al. (SC'11) define the two Weyl increments of the Philox4x32
    key schedule as the 32-bit fractional parts of the golden ratio and of
    sqrt(3): W0 = floor(2^32 (phi - 1)), W1 = floor(2^32 (sqrt(3) - 1)).
    Both are derived here with exact integer square roots, so a mistyped
    constant fails independently of any other implementation."""
    from math import isqrt
    # 2^32 (phi - 1) = (sqrt(5) 2^32 - 2^32) / 2
    w0 = (isqrt(5 << 64) - (1 << 32)) // 2
    w1 = isqrt(3 << 64) - (1 << 32)
    assert philox.W0 == w0
    assert philox.W1 == w1
    # the two multipliers must be odd: the round is then a bijection
    assert philox.M0 % 2 == 1 and philox.M1 % 2 == 1


def test_philox_is_a_bijection_on_counters():
    """For a fixed key every Philox round is invertible (odd multipliers), so
    the whole map is a permutation of the 2^128 counters: distinct counter
    blocks never produce the same four words.  Checked on 2^18 counters that
    differ in one or two words.  A round that dropped a word, or mixed the
    key in non-invertibly, would collide here with high probability."""
    n = 1 << 16
    c0 = np.arange(n, dtype=np.uint64)
    blocks = []
    for c1, c2, c3 in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]:
        w = philox.philox4x32_10(c0, c1, c2, c3, 0x1234, 0x5678)
        blocks.append(np.stack(w, axis=1))
    words = np.concatenate(blocks).view(np.dtype((np.void, 16)))
    assert np.unique(words).size == 4 * n
    # the first word alone is already (nearly) collision-free: 2^18 draws
    # from 2^32 values give about 8 birthday collisions on average
    first = np.concatenate([b[:, 0] for b in blocks])
    assert 4 * n - np.unique(first).size < 40
