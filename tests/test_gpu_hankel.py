"""a9/a10 parity: block-Hankel KRP sketches and Alg. 6 against the oracle.

Sketches: GPU (structured identity of Eq. (4.1)) vs the oracle's explicit
M (Omega1 kr Omega2), FP32 bound 1e-5.  Low-rank result: singular values
relative to sigma_1 and the reconstruction U S V^T relative to ||H||, and
exact recovery of the rank-40 Hankel of the 1024 x 1024 workload.
"""

import math

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, mat_to_dev, mat_from_dev, empty_mat, rel
from oracle import hankel as HK, philox, tensor as T
from synth import HankelSpec, hankel_config_spec, markov_parameters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


def blocks_to_dev(b, dtype):
    import torch
    m, n, nb = b.shape
    # block k column-major m x n, blocks one after another
    flat = np.concatenate([np.asfortranarray(b[:, :, k]).ravel(order="F") for k in range(nb)])
    return torch.from_numpy(flat).to(dtype).to(dev())


SPECS = [HankelSpec("small", 6, 3, 2, 9, 0.9, 5, 6, 10, 15),
         HankelSpec("odd", 10, 5, 3, 17, 0.9, 6, 10, 13, 20),
         hankel_config_spec("c4")]


@pytest.mark.parametrize("spec", SPECS, ids=[s.name for s in SPECS])
def test_hankel_sketches(ctx, spec):
    import torch
    import paper_2507_23207_gb300 as K
    b = philox.round_to_f32(markov_parameters(spec))
    o1, o2, p1, p2 = HK.sketch_factors(0, spec.s, spec.m, spec.n, spec.ell_r, spec.ell_l, "f32")
    h = HK.block_hankel(b)
    ms, ns = spec.m * spec.s, spec.n * spec.s
    y = empty_mat(ms, spec.ell_r, torch.float32)
    z = empty_mat(ns, spec.ell_l, torch.float32)
    K.krp_block_hankel_sketch(ctx, blocks_to_dev(b, torch.float32), spec.m, spec.n, spec.s,
                              mat_to_dev(o1, torch.float32), mat_to_dev(o2, torch.float32),
                              spec.ell_r, mat_to_dev(p1, torch.float32),
                              mat_to_dev(p2, torch.float32), spec.ell_l, y, z)
    torch.cuda.synchronize()
    assert rel(mat_from_dev(y, ms, spec.ell_r), h @ T.khatri_rao(o1, o2)) <= 1e-5
    assert rel(mat_from_dev(z, ns, spec.ell_l), h.T @ T.khatri_rao(p1, p2)) <= 1e-5


@pytest.mark.parametrize("spec", SPECS, ids=[s.name for s in SPECS])
def test_hankel_lowrank(ctx, spec):
    import torch
    import paper_2507_23207_gb300 as K
    b = philox.round_to_f32(markov_parameters(spec))
    ms, ns, r = spec.m * spec.s, spec.n * spec.s, spec.r
    U = empty_mat(ms, r, torch.float64)
    V = empty_mat(ns, r, torch.float64)
    S = torch.empty(r, dtype=torch.float64, device=dev())
    K.krp_block_hankel_lowrank(ctx, blocks_to_dev(b, torch.float32), spec.m, spec.n, spec.s, r,
                               spec.ell_r, spec.ell_l, 0, U, S, V)
    torch.cuda.synchronize()
    ora = HK.single_pass_svd(b, r, spec.ell_r, spec.ell_l, 0, omega_round="f32")
    h = ora["H"]
    ug, vg, sg = mat_from_dev(U, ms, r), mat_from_dev(V, ns, r), S.cpu().numpy()
    assert np.max(np.abs(sg - ora["S"])) <= 1e-5 * ora["S"][0]
    approx_g = (ug * sg) @ vg.T
    approx_o = (ora["U"] * ora["S"]) @ ora["V"].T
    assert np.linalg.norm(approx_g - approx_o) <= 1e-5 * np.linalg.norm(h)
    # exact rank (order <= r): the single-pass approximation reproduces H
    assert np.linalg.norm(h - approx_g) <= 1e-5 * np.linalg.norm(h)
    assert np.linalg.norm(ug.T @ ug - np.eye(r)) <= 1e-8


def test_hankel_host_output_and_default_ell_l(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    spec = SPECS[0]
    b = philox.round_to_f32(markov_parameters(spec))
    ms, ns, r = spec.m * spec.s, spec.n * spec.s, spec.r
    U = np.zeros((r, ms))
    V = np.zeros((r, ns))
    S = np.zeros(r)
    K.krp_block_hankel_lowrank(ctx, blocks_to_dev(b, torch.float32), spec.m, spec.n, spec.s, r,
                               spec.ell_r, 0, 0, U, S, V)
    ell_l = int(math.ceil(1.5 * spec.ell_r))
    ora = HK.single_pass_svd(b, r, spec.ell_r, ell_l, 0, omega_round="f32")
    assert np.max(np.abs(S - ora["S"])) <= 1e-5 * ora["S"][0]


def test_hankel_invalid(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    spec = SPECS[0]
    b = blocks_to_dev(philox.round_to_f32(markov_parameters(spec)), torch.float32)
    U = empty_mat(27, 6, torch.float64)
    S = torch.empty(6, dtype=torch.float64, device=dev())
    V = empty_mat(18, 6, torch.float64)
    with pytest.raises(K.KrpError) as e:  # r > ell_r
        K.krp_block_hankel_lowrank(ctx, b, 3, 2, 9, 11, 10, 15, 0, U, S, V)
    assert e.value.status == K.KRP_EINVAL
