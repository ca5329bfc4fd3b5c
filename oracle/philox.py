"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller normals.

The sketching factors Omega^(j) of a KRP (Def. of KRP, Sec. 2.5) only need
i.i.d. mean-zero unit-variance entries; the paper draws them with MATLAB's
randn.  For a reproducible, counter-addressable stream both sides of this
project implement Philox4x32 with 10 rounds from its published definition:

  round:  (c0, c1, c2, c3) ->
          (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
  key schedule: (k0, k1) += (W0, W1) between rounds
  M0 = 0xD2511F53, M1 = 0xCD9E8D57, W0 = 0x9E3779B9, W1 = 0xBB67AE85

Counter layout of a factor entry (shared contract with the device generator):
  key     = (seed mod 2^32, seed >> 32)
  counter = (e >> 2, factor index j, draw id, stream tag)
  e       = row + rows * col    (column-major element index)
Each counter yields words (w0, w1, w2, w3); entry lanes 0..3 of the block are
  z0 = rho(w0) cos(2 pi u(w1)), z1 = rho(w0) sin(2 pi u(w1)),
  z2 = rho(w2) cos(2 pi u(w3)), z3 = rho(w2) sin(2 pi u(w3)),
with u(w) = (w + 0.5) 2^-32 in (0, 1) and rho(w) = sqrt(-2 ln u(w)), in FP64.
Stream tags: 0 = Omega (right sketch), 1 = Psi (left sketch).
"""

from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

TAG_OMEGA = 0
TAG_PSI = 1


def _mulhilo(a: int, b: np.ndarray):
    prod = np.uint64(a) * b.astype(np.uint64)
    return (prod >> np.uint64(32)).astype(np.uint64), (prod & np.uint64(MASK32))


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of 32-bit counters; returns 4 uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint64) & np.uint64(MASK32)
    c1 = np.asarray(c1, dtype=np.uint64) & np.uint64(MASK32)
    c2 = np.asarray(c2, dtype=np.uint64) & np.uint64(MASK32)
    c3 = np.asarray(c3, dtype=np.uint64) & np.uint64(MASK32)
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = int(k0) & MASK32
    k1 = int(k1) & MASK32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        hi0, lo0 = _mulhilo(M0, c0)
        hi1, lo1 = _mulhilo(M1, c2)
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def factor_words(seed: int, factor: int, draw: int, tag: int, rows: int,
                 cols: int) -> np.ndarray:
    """The four Philox words of every counter block of a rows x cols factor.

    Returns an array of shape (nblocks, 4), nblocks = ceil(rows*cols/4).
    """
    n = rows * cols
    nblk = (n + 3) // 4
    blk = np.arange(nblk, dtype=np.uint64)
    w = philox4x32_10(blk, factor, draw, tag, seed & MASK32, (seed >> 32) & MASK32)
    return np.stack(w, axis=1)


def uniform_open(w: np.ndarray) -> np.ndarray:
    """u = (w + 0.5) * 2^-32, strictly inside (0, 1)."""
    return (w.astype(np.float64) + 0.5) * (2.0 ** -32)


def gaussian_factor(seed: int, factor: int, draw: int, tag: int, rows: int,
                    cols: int) -> np.ndarray:
    """rows x cols matrix of i.i.d. N(0,1) entries (FP64), entry (i,k) at e=i+rows*k."""
    words = factor_words(seed, factor, draw, tag, rows, cols)
    ua0 = uniform_open(words[:, 0])
    ub0 = uniform_open(words[:, 1])
    ua1 = uniform_open(words[:, 2])
    ub1 = uniform_open(words[:, 3])
    rho0 = np.sqrt(-2.0 * np.log(ua0))
    rho1 = np.sqrt(-2.0 * np.log(ua1))
    z = np.empty((words.shape[0], 4))
    z[:, 0] = rho0 * np.cos(2.0 * np.pi * ub0)
    z[:, 1] = rho0 * np.sin(2.0 * np.pi * ub0)
    z[:, 2] = rho1 * np.cos(2.0 * np.pi * ub1)
    z[:, 3] = rho1 * np.sin(2.0 * np.pi * ub1)
    flat = z.reshape(-1)[: rows * cols]
    return flat.reshape((rows, cols), order="F")


def round_to_f32(a: np.ndarray) -> np.ndarray:
    """Round FP64 to the nearest FP32 value (ties to even), returned as FP64."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """Round to FP32 (RN) and then to bfloat16 (RN-even), returned as FP64.

    bfloat16 keeps the top 16 bits of the FP32 pattern; rounding adds
    0x7FFF + (bit 16) before truncating.  NaN/Inf are not expected here.
    """
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    bits = (bits + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def krp_factors(seed: int, draw: int, rows, ell: int, tag: int = TAG_OMEGA,
                skip=None):
    """The factor set {Omega^(j)} of one KRP draw: Omega^(j) is rows[j] x ell.

    ``skip`` leaves out one mode (its entry is None), as in Alg. 7 and Alg. 8
    where mode i draws only the d-1 factors j != i.
    """
    out = []
    for j, nj in enumerate(rows):
        if skip is not None and j == skip:
            out.append(None)
        else:
            out.append(gaussian_factor(seed, j, draw, tag, int(nj), int(ell)))
    return out
