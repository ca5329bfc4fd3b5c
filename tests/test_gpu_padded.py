"""Padded X (per-mode leading sizes ld >= dims) and the dimension-tree split.

A padded X holds the tensor in the leading corner of a larger dense array
(element (i_1..i_d) at sum_j i_j prod_{m<j} ld_m); the padding holds other
values, which must not leak into any result.  Every entry point that takes X
gives with ld exactly the result of the same call on the dense tensor (the
library packs a dense copy first), and the oracle's within the usual bounds.
tree_split: every admissible split of the tensor-core tree (and -1, picked by
timing) gives the oracle's sketches."""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, mat_to_dev, mat_from_dev, empty_mat, rel
from oracle import philox, tensor as T, tucker as TK
from synth import TuckerSpec, tucker_tensor, to_torch_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


def _padded(x, ld, dtype, fill=7.0):
    """The tensor x (numpy, dims) in the corner of a padded device array of
    sides ld, padding = fill (torch layout (ld_d, ..., ld_1))."""
    import torch
    buf = torch.full(tuple(ld[::-1]), fill, dtype=torch.float64)
    view = buf[tuple(slice(0, n) for n in x.shape[::-1])]
    view.copy_(to_torch_layout(np.asfortranarray(x)))
    return buf.to(dtype).to(dev())


def _inputs(form, x32, dims, ld, ctx):
    import torch
    import paper_2507_23207_gb300 as K
    if form == "f32":
        return (_padded(x32, ld, torch.float32), to_torch_layout(np.asfortranarray(x32)).to(
            torch.float32).to(dev()), x32)
    if form == "bf16":
        xb = philox.round_to_bf16(x32)
        return (_padded(xb, ld, torch.bfloat16),
                to_torch_layout(np.asfortranarray(xb)).to(torch.bfloat16).to(dev()), xb)
    hi = philox.round_to_bf16(x32)
    lo = philox.round_to_bf16(x32 - hi)
    ph, pl = _padded(hi, ld, torch.bfloat16).reshape(-1), _padded(lo, ld, torch.bfloat16, 0.0).reshape(-1)
    dh = to_torch_layout(np.asfortranarray(hi)).to(torch.bfloat16).to(dev()).reshape(-1)
    dl = to_torch_layout(np.asfortranarray(lo)).to(torch.bfloat16).to(dev()).reshape(-1)
    return K.BF16x2(torch.cat([ph, pl])), K.BF16x2(torch.cat([dh, dl])), hi + lo


CASES = [((40, 23, 9), (48, 25, 11)), ((64, 20, 6, 5), (72, 20, 9, 5)), ((16, 7, 5), (16, 7, 8))]


@pytest.mark.parametrize("form", ["f32", "bf16", "bf16x2"])
@pytest.mark.parametrize("dims,ld", CASES)
def test_padded_sketches_equal_dense(ctx, form, dims, ld):
    import torch
    import paper_2507_23207_gb300 as K
    rng = np.random.default_rng(sum(dims))
    x32 = philox.round_to_f32(np.asfortranarray(rng.standard_normal(dims)))
    xp, xd, xo = _inputs(form, x32, dims, ld, ctx)
    ell = 8
    dt = torch.float32 if form == "f32" else torch.bfloat16
    om = [torch.empty((ell, n), dtype=dt, device=dev()) for n in dims]
    K.krp_gen_factors(ctx, 3, 0, 0, dims, ell, om)
    omh = [o.to(torch.float64).cpu().numpy().T for o in om]
    yp = [torch.empty((ell, n), dtype=torch.float32, device=dev()) for n in dims]
    yd = [torch.empty((ell, n), dtype=torch.float32, device=dev()) for n in dims]
    K.krp_sketch_all_modes(ctx, xp, dims, om, ell, yp, ld=ld)
    K.krp_sketch_all_modes(ctx, xd, dims, om, ell, yd)
    y0 = torch.empty((ell, dims[0]), dtype=torch.float32, device=dev())
    K.krp_sketch_mode(ctx, xp, dims, 0, om, ell, y0, ld=ld)
    torch.cuda.synchronize()
    for n in range(len(dims)):
        ref = T.mttkrp(xo, omh, n)
        got = yp[n].to(torch.float64).cpu().numpy().T
        assert rel(got, yd[n].to(torch.float64).cpu().numpy().T) <= 1e-6, (form, n)
        assert rel(got, ref) <= 1e-5, (form, n)
    assert rel(y0.to(torch.float64).cpu().numpy().T, T.mttkrp(xo, omh, 0)) <= 1e-5


@pytest.mark.parametrize("form", ["f32", "bf16"])
def test_padded_tucker_multi_ttm_and_residual(ctx, form):
    import torch
    import paper_2507_23207_gb300 as K
    spec = TuckerSpec("pad", (40, 30, 20), (4, 3, 3), 1e-3, None, 57, (4, 3, 3), (8, 7, 7))
    ld = (48, 33, 21)
    x, _, _ = tucker_tensor(spec)
    x32 = philox.round_to_f32(x)
    xp, xd, xo = _inputs(form, x32, spec.dims, ld, ctx)
    ranks = list(spec.ranks)
    flags = K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL
    outs = []
    for xx, l_ in ((xp, ld), (xd, None), (xp.cpu(), ld)):  # device padded, dense, host padded
        core = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device=dev())
        facs = [torch.empty(n * r, dtype=torch.float64, device=dev()) for n, r in zip(spec.dims, ranks)]
        res = K.krp_tucker_rhosvd(ctx, xx, spec.dims, ranks, spec.oversample, 0, flags, core, facs,
                                  ld=l_)
        torch.cuda.synchronize()
        g = core.cpu().numpy().astype(np.float64).reshape(ranks[::-1]).T
        qs = [f.cpu().numpy().reshape(r, n).T for f, n, r in zip(facs, spec.dims, ranks)]
        outs.append((g, qs, res["rel_residual"], core, facs))
    nx = np.linalg.norm(xo)
    ref = TK.reconstruct(outs[1][0], outs[1][1])
    for g, qs, e, _, _ in (outs[0], outs[2]):
        assert np.linalg.norm(TK.reconstruct(g, qs) - ref) <= 1e-6 * nx
        assert abs(e - outs[1][2]) <= 1e-4 * outs[1][2]
    # multi-TTM and residual entry points with ld
    qd = [mat_to_dev(q, torch.float64) for q in outs[1][1]]
    gp = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device=dev())
    gd = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device=dev())
    K.krp_multi_ttm(ctx, xp, spec.dims, qd, ranks, gp, ld=ld)
    K.krp_multi_ttm(ctx, xd, spec.dims, qd, ranks, gd)
    torch.cuda.synchronize()
    assert rel(gp.cpu().numpy(), gd.cpu().numpy()) <= 1e-6
    rp = K.krp_residual(ctx, xp, spec.dims, ranks, outs[1][3], outs[1][4], ld=ld)
    rd = K.krp_residual(ctx, xd, spec.dims, ranks, outs[1][3], outs[1][4])
    assert abs(rp[0] - rd[0]) <= 1e-6 * rd[0] and abs(rp[1] - rd[1]) <= 1e-6 * rd[1]


def test_padded_rejects_short_ld(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    dims = (16, 8, 4)
    x = torch.zeros(16 * 8 * 4, dtype=torch.float32, device=dev())
    om = [torch.zeros((4, n), dtype=torch.float32, device=dev()) for n in dims]
    ys = [torch.empty((4, n), dtype=torch.float32, device=dev()) for n in dims]
    with pytest.raises(K.KrpError) as e:
        K.krp_sketch_all_modes(ctx, x, dims, om, 4, ys, ld=(16, 7, 4))
    assert e.value.status == K.KRP_EINVAL


@pytest.mark.parametrize("form", ["bf16", "bf16x2"])
@pytest.mark.parametrize("dims,ell", [((64, 40, 24, 16), 12), ((200, 30, 20, 10), 30),
                                      ((128, 24, 20), 20)])
def test_every_tree_split_gives_the_oracle_sketches(ctx, form, dims, ell):
    import torch
    import paper_2507_23207_gb300 as K
    rng = np.random.default_rng(ell + sum(dims))
    x32 = philox.round_to_f32(np.asfortranarray(rng.standard_normal(dims)))
    _, xd, xo = _inputs(form, x32, dims, dims, ctx)
    om = [torch.empty((ell, n), dtype=torch.bfloat16, device=dev()) for n in dims]
    K.krp_gen_factors(ctx, 5, 0, 0, dims, ell, om)
    omh = [o.to(torch.float64).cpu().numpy().T for o in om]
    refs = [T.mttkrp(xo, omh, n) for n in range(len(dims))]
    for split in list(range(1, len(dims))) + [-1, -1]:  # -1 twice: timed, then cached
        ys = [torch.empty((ell, n), dtype=torch.float32, device=dev()) for n in dims]
        K.krp_sketch_all_modes(ctx, xd, dims, om, ell, ys, tree_split=split)
        torch.cuda.synchronize()
        for n in range(len(dims)):
            assert rel(ys[n].to(torch.float64).cpu().numpy().T, refs[n]) <= 1e-5, (split, n)
    with pytest.raises(K.KrpError) as e:
        K.krp_sketch_all_modes(ctx, xd, dims, om, ell, ys, tree_split=len(dims))
    assert e.value.status == K.KRP_EINVAL
