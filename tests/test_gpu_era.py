"""Eigensystem realization on the GPU (krp_era_realize) from the rank-r SVD of
Alg. 6 (the use Sec. 4.2 makes of the block-Hankel SVD).

For given factors (U, S, V) the state matrix A = O_top^+ H_up G^+ is unique,
so the GPU's A is compared with the oracle's era_realization run on the very
same factors (FP64 on the host): A entrywise and the eigenvalues as sets
(Hausdorff distance).  End to end, the realized eigenvalues are compared with
the system's known ones (a physical invariant of the input): on an order-8
system and on the 1024 x 1024 block Hankel of order 40, the GPU pipeline's
spectrum must agree with the oracle pipeline's on the same FP32 data within
the level of their factors (1e-5), and both must be close to the system's.
"""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, empty_mat, mat_from_dev
from tests.test_gpu_hankel import blocks_to_dev
from oracle import hankel as HK, philox
from synth import HankelSpec, hankel_config_spec, markov_parameters
from synth.hankel import system_matrices

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


def _gpu_svd_and_era(ctx, spec, b, dtype, with_a=True):
    import torch
    import paper_2507_23207_gb300 as K
    ms, ns, r = spec.m * spec.s, spec.n * spec.s, spec.r
    U = empty_mat(ms, r, torch.float64)
    V = empty_mat(ns, r, torch.float64)
    S = torch.empty(r, dtype=torch.float64, device=dev())
    bd = blocks_to_dev(b, dtype)
    K.krp_block_hankel_lowrank(ctx, bd, spec.m, spec.n, spec.s, r, spec.ell_r, spec.ell_l,
                               spec.omega_seed, U, S, V)
    A = empty_mat(r, r, torch.float64) if with_a else None
    er = torch.empty(r, dtype=torch.float64, device=dev())
    ei = torch.empty(r, dtype=torch.float64, device=dev())
    K.krp_era_realize(ctx, bd, spec.m, spec.n, spec.s, r, U, S, V, er, ei, A=A)
    torch.cuda.synchronize()
    ug, vg, sg = mat_from_dev(U, ms, r), mat_from_dev(V, ns, r), S.cpu().numpy()
    eig = er.cpu().numpy() + 1j * ei.cpu().numpy()
    return ug, sg, vg, (mat_from_dev(A, r, r) if with_a else None), eig


SPECS = [HankelSpec("era8", 8, 3, 3, 14, 0.9, 21, r=8, ell_r=12, ell_l=18),
         HankelSpec("era12", 12, 4, 2, 30, 0.95, 33, r=12, ell_r=20, ell_l=30),
         hankel_config_spec("c4")]


@pytest.mark.parametrize("spec", SPECS, ids=[s.name for s in SPECS])
def test_era_matches_oracle_and_system(ctx, spec):
    import torch
    b = philox.round_to_f32(markov_parameters(spec))
    ug, sg, vg, ag, eg = _gpu_svd_and_era(ctx, spec, b, torch.float32)
    # the same factors through the oracle's realization (FP64, least squares)
    a_o = HK.era_realization(b, ug, sg, vg)
    assert np.linalg.norm(ag - a_o) <= 1e-10 * np.linalg.norm(a_o)
    e_o = np.linalg.eigvals(a_o)
    assert HK.hausdorff(eg, e_o) <= 1e-10 * np.max(np.abs(e_o))
    # conjugate pairs adjacent, positive imaginary part first
    im = eg.imag
    i = 0
    while i < len(eg):
        if im[i] != 0:
            assert im[i] > 0 and eg[i + 1] == np.conj(eg[i])
            i += 2
        else:
            i += 1
    # end to end: the distance to the system's eigenvalues is the oracle
    # pipeline's (Alg. 6 + realization on the same FP32 blocks), both limited
    # by the FP32 rounding of the data
    _, _, _, eig_true = system_matrices(spec)
    ora = HK.single_pass_svd(b, spec.r, spec.ell_r, spec.ell_l, spec.omega_seed, omega_round="f32")
    h_ora = HK.hausdorff(np.linalg.eigvals(HK.era_realization(b, ora["U"], ora["S"], ora["V"])),
                         eig_true)
    h_gpu = HK.hausdorff(eg, eig_true)
    # the two pipelines' spectra agree at the level of their factors (P2:
    # U S V^T within 1e-5 of ||H||, the eigenvalues of these normal systems
    # well conditioned), so by the triangle inequality of the Hausdorff
    # distance h_gpu <= h_ora + that agreement
    e_pipe = np.linalg.eigvals(HK.era_realization(b, ora["U"], ora["S"], ora["V"]))
    agree = HK.hausdorff(eg, e_pipe)
    assert agree <= 1e-5 * np.max(np.abs(eig_true)), agree
    assert h_gpu <= h_ora + agree + 1e-15, (h_gpu, h_ora, agree)
    assert h_gpu <= 1e-4, h_gpu
    print(f"{spec.name}: hausdorff to the system's eigenvalues gpu {h_gpu:.2e}, oracle {h_ora:.2e}")


def test_era_without_a_and_bf16_blocks(ctx):
    import torch
    spec = SPECS[0]
    b = philox.round_to_bf16(markov_parameters(spec))
    ug, sg, vg, _, eg = _gpu_svd_and_era(ctx, spec, b, torch.bfloat16, with_a=False)
    e_o = np.linalg.eigvals(HK.era_realization(b, ug, sg, vg))
    assert HK.hausdorff(eg, e_o) <= 1e-10 * np.max(np.abs(e_o))


def test_era_invalid(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    spec = SPECS[0]
    r = spec.r
    bd = blocks_to_dev(philox.round_to_f32(markov_parameters(spec)), torch.float32)
    U = empty_mat(spec.m * spec.s, r, torch.float64)
    V = empty_mat(spec.n * spec.s, r, torch.float64)
    S = torch.ones(r, dtype=torch.float64, device=dev())
    e = torch.empty(r, dtype=torch.float64, device=dev())
    with pytest.raises(K.KrpError) as ex:  # r > 64
        K.krp_era_realize(ctx, bd, spec.m, spec.n, spec.s, 65, U, S, V, e, e)
    assert ex.value.status == K.KRP_EINVAL
    with pytest.raises(K.KrpError) as ex:  # host buffers
        K.krp_era_realize(ctx, bd, spec.m, spec.n, spec.s, r, U, S, V, e.cpu(), e)
    assert ex.value.status == K.KRP_EINVAL
