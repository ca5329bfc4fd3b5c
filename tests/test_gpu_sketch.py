"""a2/a3 parity: KRP sketches on the GPU against the oracle's explicit-KRP MTTKRP.

Both sides see the same FP32-rounded X and the same factors (drawn by the
oracle's own Philox and uploaded).  FP32 bound: relative Frobenius error
<= 1e-5 per sketch.  Shapes span several 128-row tiles, ragged tails, a
size-1 mode, d = 2, 3, 4.
"""

import numpy as np
import pytest

from tests.gpu_util import (require_gpu, dev, mat_to_dev, mat_from_dev, empty_mat,
                            tensor_to_dev, rel)
from oracle import philox, tensor as T

pytestmark = pytest.mark.gpu

CASES = [((37, 29, 23), 5), ((37, 29, 23), 1), ((16, 8, 4, 6), 7), ((130, 70, 33), 48),
         ((3, 2), 2), ((5, 1, 7), 3), ((129, 65, 3), 13), ((64, 64, 64), 10),
         ((200, 9, 11, 3), 30), ((257, 33, 17), 64), ((20, 30, 40), 100)]


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


def make_case(dims, ell, seed=11, xform="f32"):
    rng = np.random.default_rng(seed + sum(dims) + ell)
    x = np.asfortranarray(rng.standard_normal(dims))
    x = philox.round_to_f32(x) if xform == "f32" else philox.round_to_bf16(x)
    rnd = philox.round_to_f32 if xform == "f32" else philox.round_to_bf16
    om = [rnd(philox.gaussian_factor(5, j, 0, 0, n, ell)) for j, n in enumerate(dims)]
    return x, om


@pytest.mark.parametrize("dims,ell", CASES)
def test_sketch_mode_f32(ctx, dims, ell):
    import torch
    import paper_2507_23207_gb300 as K
    x, om = make_case(dims, ell)
    xd = tensor_to_dev(x, torch.float32)
    omd = [mat_to_dev(o, torch.float32) for o in om]
    for n in range(len(dims)):
        y = empty_mat(dims[n], ell, torch.float32)
        K.krp_sketch_mode(ctx, xd, dims, n, omd, ell, y)
        torch.cuda.synchronize()
        ref = T.mttkrp(x, om, n)
        assert rel(mat_from_dev(y, dims[n], ell), ref) <= 1e-5, (dims, n)


@pytest.mark.parametrize("dims,ell", CASES)
def test_sketch_all_modes_f32(ctx, dims, ell):
    import torch
    import paper_2507_23207_gb300 as K
    x, om = make_case(dims, ell, seed=3)
    xd = tensor_to_dev(x, torch.float32)
    omd = [mat_to_dev(o, torch.float32) for o in om]
    ys = [empty_mat(n, ell, torch.float32) for n in dims]
    K.krp_sketch_all_modes(ctx, xd, dims, omd, ell, ys)
    torch.cuda.synchronize()
    for n in range(len(dims)):
        ref = T.mttkrp(x, om, n)
        assert rel(mat_from_dev(ys[n], dims[n], ell), ref) <= 1e-5, (dims, n)


def test_sketch_with_device_generated_factors(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    dims, ell = (48, 40, 36), 12
    x, om = make_case(dims, ell, seed=8)
    xd = tensor_to_dev(x, torch.float32)
    omd = [empty_mat(n, ell, torch.float32) for n in dims]
    K.krp_gen_factors(ctx, 5, 0, 0, dims, ell, omd)
    ys = [empty_mat(n, ell, torch.float32) for n in dims]
    K.krp_sketch_all_modes(ctx, xd, dims, omd, ell, ys)
    torch.cuda.synchronize()
    for n in range(3):
        assert rel(mat_from_dev(ys[n], dims[n], ell), T.mttkrp(x, om, n)) <= 1e-5


def test_sketch_invalid_arguments(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    dims, ell = (8, 8, 8), 4
    x, om = make_case(dims, ell)
    xd = tensor_to_dev(x, torch.float32)
    omd = [mat_to_dev(o, torch.float32) for o in om]
    y = empty_mat(8, ell, torch.float32)
    for bad in [dict(n=3), dict(n=-1)]:
        with pytest.raises(K.KrpError) as e:
            K.krp_sketch_mode(ctx, xd, dims, bad["n"], omd, ell, y)
        assert e.value.status == K.KRP_EINVAL
    with pytest.raises(K.KrpError):
        K.krp_sketch_mode(ctx, xd, dims, 0, omd, 0, y)
    with pytest.raises(K.KrpError):  # factor dtype must match X dtype
        K.krp_sketch_mode(ctx, xd, dims, 0, [o.to(torch.bfloat16) for o in omd], ell, y)
    with pytest.raises(K.KrpError):
        K.krp_sketch_mode(ctx, xd, [8], 0, omd, ell, y)
    assert "out of range" in ctx.last_error() or ctx.last_error() != ""
