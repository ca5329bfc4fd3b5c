"""Recompression of the Hadamard (elementwise) product of two Tucker tensors
with KRP sketches (Sec. 5, its opening: the randomized HOSVD of Kressner and
Perisa with Khatri-Rao sketching matrices), FP64 on the host.

Test-infrastructure only: the CUDA library never imports this module.

The oracle forms the product explicitly, Z = X * Y with X = G x {U_i} and
Y = H x {V_i}, and runs RHOSVD-KRP-MEMO (Alg. 7 with one factor set) on it.
"""

from __future__ import annotations

from typing import Sequence

import numpy as np

from .tucker import reconstruct, rhosvd_krp, rel_error


def hadamard_of_tucker(g: np.ndarray, us: Sequence[np.ndarray], h: np.ndarray,
                       vs: Sequence[np.ndarray]) -> np.ndarray:
    """Z = (G x {U_i}) * (H x {V_i}), elementwise, formed explicitly."""
    return reconstruct(g, us) * reconstruct(h, vs)


def rhosvd_krp_hadamard(g, us, h, vs, ell: int, seed: int):
    """RHOSVD-KRP-MEMO of the explicit product, l = ell in every mode, FP64
    factors; returns the oracle's dict plus Z and the relative error."""
    z = hadamard_of_tucker(g, us, h, vs)
    out = rhosvd_krp(z, [ell] * z.ndim, seed, memo=True)
    out["Z"] = z
    out["rel_error"] = rel_error(z, out["G"], out["Q"])
    return out
