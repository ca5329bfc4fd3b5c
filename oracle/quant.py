"""FP8 E4M3 storage of a tensor with one scale per slab of its slowest mode.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper streams X in one working precision; a random projection only has to
capture the range of X, so a coarser storage format is a natural option for
the sketch.  This module fixes, in FP64 by definition, what an FP8 E4M3 copy
of X holds, so that a device form can be compared with it code for code:

  E4M3 ("fn" variant, OCP 8-bit floating point): sign bit, 4 exponent bits
  with bias 7, 3 mantissa bits, no infinities; code 0x7F / 0xFF is NaN.
    exponent field e > 0:  (-1)^s 2^(e-7) (1 + m/8)
    exponent field e = 0:  (-1)^s 2^(-6) (m/8)          (subnormals)
  largest finite value 2^8 (1 + 6/8) = 448, smallest subnormal 2^-9.

  Rounding: round to nearest, ties to the even code (mantissa LSB 0), with
  saturation to +-448 for finite values beyond the range ("satfinite").

  Slab scales: slab t is X[..., t] (one index of the slowest mode, i.e. one
  contiguous block of the mode-1-fastest layout).  Its scale is
  s_t = fl32(amax_t / 448), amax_t = max |fl32(X[..., t])|, so that the
  largest entry of the slab maps to the top of the E4M3 range.  A slab whose
  scale is 0 (all zero, or amax below 448 times the smallest FP32 subnormal)
  takes s_t = 1.  The code of an entry is the E4M3 rounding of the FP32
  quotient fl32(x / s_t): the quotient is taken in FP32 because that is the
  precision in which a device kernel takes the same integer decision.
  The stored value is x~ = q * s_t, exact in FP64 (4 + 24 significant bits).
"""

from __future__ import annotations

import numpy as np

E4M3_MAX = 448.0
E4M3_MIN_SUBNORMAL = 2.0 ** -9
E4M3_MIN_NORMAL = 2.0 ** -6


def e4m3_decode(codes) -> np.ndarray:
    """FP64 value of each E4M3 byte code (NaN for 0x7F and 0xFF)."""
    c = np.asarray(codes, dtype=np.int64) & 0xFF
    sign = np.where(c >> 7, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = (c & 0x7).astype(np.float64)
    mag = np.where(e == 0, np.ldexp(m / 8.0, -6), np.ldexp(1.0 + m / 8.0, e - 7))
    out = sign * mag
    return np.where((c & 0x7F) == 0x7F, np.nan, out)


def _positive_grid() -> np.ndarray:
    """The finite non-negative E4M3 values in code order 0x00..0x7E (ascending)."""
    return e4m3_decode(np.arange(0x7F))


def round_to_e4m3_codes(a) -> np.ndarray:
    """E4M3 codes of the FP32 values of ``a``: RN-even, saturating finite overflow.

    ``a`` is rounded to FP32 first (the values a device kernel converts).
    Returns uint8 codes; NaN maps to 0x7F.
    """
    v = np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)
    grid = _positive_grid()
    mag = np.abs(v)
    codes = np.empty(v.shape, dtype=np.int64)
    sat = mag >= E4M3_MAX
    codes[sat] = 0x7E
    rest = ~sat & ~np.isnan(v)
    x = mag[rest]
    lo = np.searchsorted(grid, x, side="right") - 1       # grid[lo] <= x < grid[lo + 1]
    d_lo = x - grid[lo]
    d_hi = grid[lo + 1] - x
    pick_hi = (d_hi < d_lo) | ((d_hi == d_lo) & (lo % 2 == 1))
    codes[rest] = lo + pick_hi
    codes[np.isnan(v)] = 0x7F
    neg = (v < 0) | ((v == 0) & np.signbit(v))
    codes = np.where(neg, codes | 0x80, codes)
    return codes.astype(np.uint8)


def round_to_e4m3(a) -> np.ndarray:
    """FP64 values of the E4M3 rounding of the FP32 values of ``a``."""
    return e4m3_decode(round_to_e4m3_codes(a))


def slab_scales(x: np.ndarray) -> np.ndarray:
    """s_t = fl32(max |fl32(X[..., t])| / 448) per slab of the last axis (1 where that is 0)."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    axes = tuple(range(x32.ndim - 1))
    amax = np.max(np.abs(x32), axis=axes) if axes else np.abs(x32)
    s = (amax / np.float32(E4M3_MAX)).astype(np.float32)
    s = np.where(s == 0, np.float32(1.0), s)
    return s.astype(np.float64)


def quantize_slabs(x: np.ndarray):
    """E4M3 codes of X with per-slab scales: returns (codes uint8, scales FP64).

    codes[..., t] = E4M3(fl32(fl32(X[..., t]) / s_t)), the division in FP32.
    """
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    s = slab_scales(x).astype(np.float32)
    quot = x32 / s                      # FP32 division, broadcast over the last axis
    return round_to_e4m3_codes(quot), s.astype(np.float64)


def dequantize_slabs(codes: np.ndarray, scales: np.ndarray) -> np.ndarray:
    """x~ = q * s_t in FP64 (exact: at most 4 + 24 significant bits)."""
    return e4m3_decode(codes) * np.asarray(scales, dtype=np.float64)
