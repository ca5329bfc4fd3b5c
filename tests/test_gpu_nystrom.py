"""NEXT-1: the Nystrom approximation of an SPSD block Hankel matrix (Sec. 4.1,
the remark after Alg. 6) against the oracle's explicit FP64 computation.

Inputs: symmetric systems (A = A^T, C = B^T), so M = K^T K is SPSD of rank
<= order; blocks rounded to FP32 or BF16 and factors rounded alike, the
oracle run on the same rounded values.  The pseudoinverse's cut-off rcond is
taken, per case, where the oracle's spectrum of Omega^T M Omega has no
eigenvalue within 20% of rcond * c_1, so that the two sides keep the same
eigenvalues (the CUDA path's C differs by the FP32 sketch's rounding,
~1e-6 c_1, inside that gap for rcond >= 1e-5).
Checks: eigenvalues within 1e-5 Lambda_1; U Lambda U^T within 1e-5 ||M||_F;
U orthonormal to 1e-10; for FP32 blocks, M - U Lambda U^T positive
semidefinite to 1e-5 ||M|| (the Loewner bound M_nys <= M of an SPSD M, at any
size; BF16 rounding of the blocks leaves M indefinite at ~2^-9 ||M||).  Measured differences on
these inputs are ~1e-6 (an FP32 rounding model of Y gives 5e-7).
"""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, mat_from_dev, empty_mat
from tests.test_gpu_hankel import blocks_to_dev
from oracle import hankel as HK, philox
from synth import HankelSpec, symmetric_markov_parameters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


# (name, order, m, s, radius, seed, r, ell): exact rank (order <= ell), a sketch
# smaller than the rank, and the 1024 x 1024 size of the block Hankel workload
CASES = [("exact", 6, 3, 9, 0.9, 31, 6, 10), ("deficient", 12, 4, 16, 0.9, 32, 5, 8),
         ("mid", 20, 8, 64, 0.9, 33, 16, 30), ("c4size", 40, 8, 128, 0.95, 34, 32, 50)]


def _pick_rcond(c):
    """The smallest cut-off >= 1e-5 with no eigenvalue ratio c_i / c_1 within
    20% of it (the CUDA path's C is off by ~1e-6 c_1, under 20% of any such
    cut-off, so both sides keep the same eigenvalues)."""
    ratio = np.sort(np.linalg.eigvalsh(c))[::-1]
    ratio = ratio / ratio[0]
    for rc in np.geomspace(1e-5, 1e-2, 31):
        if not np.any(np.abs(ratio - rc) <= 0.2 * rc):
            return float(rc)
    raise AssertionError("no eigenvalue gap for the cut-off")


@pytest.mark.parametrize("form", ["f32", "bf16"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_nystrom_matches_oracle(ctx, case, form):
    import torch
    import paper_2507_23207_gb300 as K
    name, order, m, s, radius, seed, r, ell = case
    spec = HankelSpec(name, order, m, m, s, radius, seed, r, ell, ell)
    b = symmetric_markov_parameters(spec)
    b = philox.round_to_f32(b) if form == "f32" else philox.round_to_bf16(b)
    dtype = torch.float32 if form == "f32" else torch.bfloat16
    probe = HK.nystrom(b, r, ell, 0, omega_round=form)
    rc = _pick_rcond(probe["C"])
    ora = HK.nystrom(b, r, ell, 0, rcond=rc, omega_round=form)
    assert ora["kept"] >= r
    ms = m * s
    U = empty_mat(ms, r, torch.float64)
    L = torch.empty(r, dtype=torch.float64, device=dev())
    K.krp_block_hankel_nystrom(ctx, blocks_to_dev(b, dtype), m, s, r, ell, 0, U, L, rcond=rc)
    torch.cuda.synchronize()
    ug, lg = mat_from_dev(U, ms, r), L.cpu().numpy()
    h = ora["H"]
    nh = np.linalg.norm(h)
    assert np.max(np.abs(lg - ora["L"])) <= 1e-5 * ora["L"][0], (lg[:4], ora["L"][:4])
    approx_g = (ug * lg) @ ug.T
    approx_o = (ora["U"] * ora["L"]) @ ora["U"].T
    assert np.linalg.norm(approx_g - approx_o) <= 1e-5 * nh
    assert np.linalg.norm(ug.T @ ug - np.eye(r)) <= 1e-10
    if form == "f32":  # BF16 rounding of the blocks leaves M indefinite at ~2^-9 ||M||
        assert np.linalg.eigvalsh(h - approx_g).min() >= -1e-5 * nh


def test_nystrom_default_cutoff_and_host_buffers(ctx):
    """rcond = 0 selects the documented 1e-5; host blocks and outputs are
    staged like krp_block_hankel_lowrank's."""
    import torch
    import paper_2507_23207_gb300 as K
    spec = HankelSpec("host", 8, 4, 4, 12, 0.9, 36, 6, 12, 12)  # C spectrum: no c_i / c_1 in [3e-6, 3e-5]
    b = philox.round_to_f32(symmetric_markov_parameters(spec))
    ora = HK.nystrom(b, 6, 12, 7, omega_round="f32")
    ms = 4 * 12
    U = torch.empty((6, ms), dtype=torch.float64).pin_memory()
    L = torch.empty(6, dtype=torch.float64).pin_memory()
    K.krp_block_hankel_nystrom(ctx, blocks_to_dev(b, torch.float32).cpu(), 4, 12, 6, 12, 7, U, L)
    ug = U.numpy().T
    assert np.max(np.abs(L.numpy() - ora["L"])) <= 1e-5 * ora["L"][0]
    assert np.linalg.norm((ug * L.numpy()) @ ug.T - (ora["U"] * ora["L"]) @ ora["U"].T) <= \
        1e-5 * np.linalg.norm(ora["H"])


def test_nystrom_rejects_bad_arguments(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    spec = HankelSpec("bad", 6, 3, 3, 9, 0.9, 36, 6, 10, 10)
    bd = blocks_to_dev(philox.round_to_f32(symmetric_markov_parameters(spec)), torch.float32)
    U = empty_mat(27, 6, torch.float64)
    L = torch.empty(6, dtype=torch.float64, device=dev())
    for r, ell, rc in ((7, 6, 0.0), (6, 65, 0.0), (6, 10, 1.0)):
        with pytest.raises(K.KrpError) as e:
            K.krp_block_hankel_nystrom(ctx, bd, 3, 9, r, ell, 0, U, L, rcond=rc)
        assert e.value.status == K.KRP_EINVAL
