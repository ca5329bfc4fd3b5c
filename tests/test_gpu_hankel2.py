"""NEXT-3: Alg. 6 on two-level block Hankel matrices (Sec. 4.3, multilevel
structure) against the oracle's explicit computation.

Inputs are two-dimensional exponential sums (rank <= order), FP32 or BF16
blocks, factors rounded alike; the oracle forms M and the three-factor
Khatri-Rao sketches explicitly.  Checks as for one level: singular values
within 1e-5 sigma_1, U S V^T within 1e-5 ||M||; exact recovery of M when
order <= r; orthonormal columns of U (to 2e-5) for the singular values the
Gram-based SVD of W resolves (sigma_j >= 1e-3 sigma_1).  Under FP32-level perturbations of the blocks the oracle's own
result moves by ~3e-7 ||M|| on these inputs.
"""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, empty_mat, mat_from_dev
from oracle import hankel as HK, philox
from synth import two_level_markov_parameters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


# (order, m, n, s1, s2, r, l_r, l_l): exact rank; truncated (r < order);
# rank above l_r; a 1024 x 1024 matrix (16 x 16 blocks of 16 x 16 blocks of 4 x 4)
CASES = [(5, 3, 2, 6, 5, 5, 9, 14), (12, 4, 4, 8, 16, 10, 20, 30), (16, 3, 3, 6, 6, 6, 10, 15),
         (20, 4, 4, 16, 16, 20, 30, 45)]


def _to_dev(b, dtype):
    import torch
    return torch.from_numpy(np.asfortranarray(b).ravel(order="F").copy()).to(dtype).to(dev())


@pytest.mark.parametrize("form", ["f32", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=[f"o{c[0]}_{c[3]}x{c[4]}" for c in CASES])
def test_two_level_lowrank(ctx, case, form):
    import torch
    import paper_2507_23207_gb300 as K
    order, m, n, s1, s2, r, lr, ll = case
    b = two_level_markov_parameters(order, m, n, s1, s2, seed=7)
    b = philox.round_to_f32(b) if form == "f32" else philox.round_to_bf16(b)
    dtype = torch.float32 if form == "f32" else torch.bfloat16
    ms, ns = m * s1 * s2, n * s1 * s2
    U = empty_mat(ms, r, torch.float64)
    V = empty_mat(ns, r, torch.float64)
    S = torch.empty(r, dtype=torch.float64, device=dev())
    K.krp_block_hankel2_lowrank(ctx, _to_dev(b, dtype), m, n, s1, s2, r, lr, ll, 0, U, S, V)
    torch.cuda.synchronize()
    ora = HK.single_pass_svd2(b, r, lr, ll, 0, omega_round=form)
    h = ora["H"]
    ug, vg, sg = mat_from_dev(U, ms, r), mat_from_dev(V, ns, r), S.cpu().numpy()
    assert np.max(np.abs(sg - ora["S"])) <= 1e-5 * ora["S"][0]
    approx_g = (ug * sg) @ vg.T
    approx_o = (ora["U"] * ora["S"]) @ ora["V"].T
    assert np.linalg.norm(approx_g - approx_o) <= 1e-5 * np.linalg.norm(h)
    # U = Q U_W with U_W the eigenvectors of W W^T (FP32 Jacobi, two FP64
    # refinement steps): on a graded spectrum (sigma_20 / sigma_1 = 2.7e-3 on
    # the 1024 x 1024 case, a Gram eigenvalue ratio of 7e-6) the columns of the
    # small singular values are orthonormal to ~7e-6 (measured); below
    # 1e-3 sigma_1 they are not resolved
    k = int(np.sum(sg >= 1e-3 * sg[0]))
    assert np.linalg.norm(ug[:, :k].T @ ug[:, :k] - np.eye(k)) <= 2e-5
    if order <= r and form == "f32":
        assert np.linalg.norm(approx_g - h) <= 1e-5 * np.linalg.norm(h)


def test_two_level_rejects_bad_arguments(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    b = _to_dev(philox.round_to_f32(two_level_markov_parameters(3, 2, 2, 3, 3, seed=1)),
                torch.float32)
    U = empty_mat(18, 3, torch.float64)
    V = empty_mat(18, 3, torch.float64)
    S = torch.empty(3, dtype=torch.float64, device=dev())
    for r, lr, ll in ((4, 3, 5), (3, 65, 70), (3, 19, 20)):
        with pytest.raises(K.KrpError) as e:
            K.krp_block_hankel2_lowrank(ctx, b, 2, 2, 3, 3, r, lr, ll, 0, U, S, V)
        assert e.value.status == K.KRP_EINVAL
