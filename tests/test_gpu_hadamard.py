"""NEXT-4: recompression of the Hadamard product of two Tucker tensors
(Sec. 5, its opening) on the GPU, structured (the product is never formed),
against the oracle's RHOSVD-KRP-MEMO of the explicit product.

Both sides are FP64 with the same Philox factors, so the reconstructions
agree to ~1e-12 of ||Z|| (checked at 1e-9, basis-invariant through
tests/parity.recon_distance) and the error values to 1e-8 absolute (the
library evaluates e from ||Z||^2 - ||core||^2, whose cancellation floor is
~1e-8 for e near 0; exact-rank cases are checked against that floor).
"""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, tensor_to_dev, mat_to_dev, mat_from_dev
from tests.parity import recon_distance
from oracle import hadamard as HD
from synth import haar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


CASES = [((40, 36, 30), (4, 3, 5), (3, 4, 2), 10), ((40, 36, 30), (2, 2, 2), (2, 3, 2), 6),
         ((12, 10, 9, 8), (2, 2, 2, 2), (2, 2, 1, 2), 4), ((60, 50, 40), (5, 4, 6), (4, 5, 3), 16)]


def _pair(dims, r, s, seed):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(r)
    h = rng.standard_normal(s)
    us = [haar(n, k, rng) for n, k in zip(dims, r)]
    vs = [haar(n, k, rng) for n, k in zip(dims, s)]
    return g, us, h, vs


@pytest.mark.parametrize("case", CASES, ids=[f"d{len(c[0])}_l{c[3]}" for c in CASES])
def test_hadamard_matches_oracle(ctx, case):
    import torch
    import paper_2507_23207_gb300 as K
    dims, r, s, ell = case
    g, us, h, vs = _pair(dims, r, s, 800 + ell)
    d = len(dims)
    core = torch.empty(ell ** d, dtype=torch.float64, device=dev())
    facs = [torch.empty((ell, n), dtype=torch.float64, device=dev()) for n in dims]
    e_gpu = K.krp_tucker_hadamard(ctx, dims, r, tensor_to_dev(g, torch.float64),
                                  [mat_to_dev(u, torch.float64) for u in us], s,
                                  tensor_to_dev(h, torch.float64),
                                  [mat_to_dev(v, torch.float64) for v in vs], ell, 3, core, facs)
    torch.cuda.synchronize()
    qs = [mat_from_dev(f, n, ell) for f, n in zip(facs, dims)]
    gz = core.cpu().numpy().reshape((ell,) * d, order="F")
    ora = HD.rhosvd_krp_hadamard(g, us, h, vs, ell, 3)
    nz = np.linalg.norm(ora["Z"])
    for q in qs:
        assert np.linalg.norm(q.T @ q - np.eye(ell)) <= 1e-12
    assert recon_distance(gz, qs, ora["G"], ora["Q"]) <= 1e-9 * nz
    assert abs(e_gpu - ora["rel_error"]) <= 1e-8, (e_gpu, ora["rel_error"])
    full_rank = all(ell >= a * b for a, b in zip(r, s))
    if full_rank:
        assert e_gpu <= 1e-7


def test_hadamard_rejects_bad_arguments(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    dims, r, s = (10, 9, 8), (2, 2, 2), (2, 2, 2)
    g, us, h, vs = _pair(dims, r, s, 1)
    G, H = tensor_to_dev(g, torch.float64), tensor_to_dev(h, torch.float64)
    U = [mat_to_dev(u, torch.float64) for u in us]
    V = [mat_to_dev(v, torch.float64) for v in vs]
    core = torch.empty(1000, dtype=torch.float64, device=dev())
    facs = [torch.empty(n * 10, dtype=torch.float64, device=dev()) for n in dims]
    for ell in (0, 9, 65):
        with pytest.raises(K.KrpError) as e:
            K.krp_tucker_hadamard(ctx, dims, r, G, U, s, H, V, ell, 0, core, facs)
        assert e.value.status == K.KRP_EINVAL
