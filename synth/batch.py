"""Seeded batches of small, uneven problems (the batched workload).

Tensors: each of the three sides uniform in 32..192 and each multilinear rank
uniform in 4..16, drawn independently per mode; core N(0,1), Haar factors,
relative noise 1e-5; sketch size l_i = r_i + 8.  Block Hankel matrices: state
order uniform over the even values in 8..32, square blocks of side uniform in
4..8, block rows s uniform in 32..128, target rank = order, l_r = order + 8,
l_l = ceil(1.5 l_r).  Item b of the tensor batch uses data seed 1005 + b and
Philox key b.  Input construction only.
"""

from __future__ import annotations

import math
from typing import List

import numpy as np

from .hankel import HankelSpec
from .tucker import TuckerSpec


def batch_tucker_specs(count: int = 512, seed: int = 1005, sides=(32, 192), ranks=(4, 16),
                       noise: float = 1e-5, oversample: int = 8) -> List[TuckerSpec]:
    rng = np.random.default_rng([seed, 5])
    out = []
    for b in range(count):
        dims = tuple(int(v) for v in rng.integers(sides[0], sides[1] + 1, 3))
        rk = tuple(int(v) for v in rng.integers(ranks[0], ranks[1] + 1, 3))
        ell = tuple(r + oversample for r in rk)
        out.append(TuckerSpec(f"batch-{b}", dims, rk, noise, None, seed + b, rk, ell,
                              omega_seed=b))
    return out


def batch_hankel_specs(count: int = 64, seed: int = 1005, orders=(8, 32), blocks=(4, 8),
                       block_rows=(32, 128), oversample: int = 8) -> List[HankelSpec]:
    rng = np.random.default_rng([seed, 6])
    out = []
    for b in range(count):
        order = 2 * int(rng.integers(orders[0] // 2, orders[1] // 2 + 1))
        m = int(rng.integers(blocks[0], blocks[1] + 1))
        s = int(rng.integers(block_rows[0], block_rows[1] + 1))
        ell_r = order + oversample
        out.append(HankelSpec(f"hbatch-{b}", order, m, m, s, 0.95, seed + 100 + b, order, ell_r,
                              int(math.ceil(1.5 * ell_r)), omega_seed=b))
    return out
