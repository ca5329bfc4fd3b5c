"""BF16 tensor-core (tcgen05) path: parity against the oracle on BF16-rounded data.

The oracle sees exactly the BF16 values the GPU streams (X and factors rounded
RN-even from FP32), so products are exact on both sides and only FP32
accumulation differs: sketches keep the 1e-5 bound.  The core uses Q_1 split
into a BF16 hi/lo pair (|Q - hi - lo| <= 2^-17 |Q|), so the core and the
reconstruction get a bound derived from that split: 3e-5 (core, relative) and
5e-5 (reconstruction relative to ||X||).
"""

import numpy as np
import pytest

from tests.gpu_util import (require_gpu, dev, mat_to_dev, mat_from_dev, empty_mat,
                            tensor_to_dev, tensor_from_dev, rel)
from oracle import linalg as L, philox, tensor as T, tucker as TK
from tests.parity import U_BF16_PAIR, check_error_value, eval_bound
from synth import TuckerSpec, tucker_tensor

pytestmark = pytest.mark.gpu

# (1024, 64, 5) at l = 48 and (1024, 40, 6) at l = 64 cut i1 into two and
# three segments of the one-pass tree (the last one short)
CASES = [((64, 48, 40), 5), ((128, 72, 33), 16), ((200, 200, 7), 30), ((256, 64, 16, 3), 12),
         ((1024, 64, 5), 48), ((136, 40, 30), 64), ((8, 9, 10), 3), ((520, 130, 9), 20),
         ((1024, 40, 6), 64)]


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


def bf16_case(dims, ell, seed=1):
    rng = np.random.default_rng(seed + sum(dims) + ell)
    x = philox.round_to_bf16(np.asfortranarray(rng.standard_normal(dims)))
    om = [philox.round_to_bf16(philox.gaussian_factor(9, j, 0, 0, n, ell))
          for j, n in enumerate(dims)]
    return x, om


@pytest.mark.parametrize("dims,ell", CASES)
def test_bf16_sketch_mode(ctx, dims, ell):
    import torch
    import paper_2507_23207_gb300 as K
    x, om = bf16_case(dims, ell)
    xd = tensor_to_dev(x, torch.bfloat16)
    omd = [mat_to_dev(o, torch.bfloat16) for o in om]
    for n in range(len(dims)):
        y = empty_mat(dims[n], ell, torch.float32)
        K.krp_sketch_mode(ctx, xd, dims, n, omd, ell, y)
        torch.cuda.synchronize()
        assert rel(mat_from_dev(y, dims[n], ell), T.mttkrp(x, om, n)) <= 1e-5, (dims, n)


@pytest.mark.parametrize("dims,ell", CASES)
def test_bf16_sketch_all_modes(ctx, dims, ell):
    import torch
    import paper_2507_23207_gb300 as K
    x, om = bf16_case(dims, ell, seed=2)
    xd = tensor_to_dev(x, torch.bfloat16)
    omd = [mat_to_dev(o, torch.bfloat16) for o in om]
    ys = [empty_mat(n, ell, torch.float32) for n in dims]
    K.krp_sketch_all_modes(ctx, xd, dims, omd, ell, ys)
    torch.cuda.synchronize()
    for n in range(len(dims)):
        assert rel(mat_from_dev(ys[n], dims[n], ell), T.mttkrp(x, om, n)) <= 1e-5, (dims, n)


@pytest.mark.parametrize("dims,cols", [((64, 48, 40), (8, 6, 5)), ((1024, 64, 5), (48, 20, 5)),
                                       ((200, 40, 30, 7), (30, 10, 9, 7)), ((16, 16, 16), (16, 16, 16))])
def test_bf16_multi_ttm(ctx, dims, cols):
    import torch
    import paper_2507_23207_gb300 as K
    rng = np.random.default_rng(5)
    x = philox.round_to_bf16(np.asfortranarray(rng.standard_normal(dims)))
    qs = [L.householder_qr(rng.standard_normal((n, c)))[0] for n, c in zip(dims, cols)]
    g = torch.empty(int(np.prod(cols)), dtype=torch.float32, device=dev())
    K.krp_multi_ttm(ctx, tensor_to_dev(x, torch.bfloat16), dims, [mat_to_dev(q, torch.float64) for q in qs],
                    cols, g)
    torch.cuda.synchronize()
    assert rel(tensor_from_dev(g, cols), T.multi_ttm(x, [q.T for q in qs])) <= 3e-5


SPECS = [TuckerSpec("b1", (64, 48, 40), (4, 4, 4), 1e-3, None, 41, (4, 4, 4), (8, 8, 8)),
         TuckerSpec("b2", (128, 40, 24, 16), (3, 3, 3, 3), 1e-2, None, 43, (3, 3, 3, 3), (6, 6, 6, 6))]


@pytest.mark.parametrize("spec", SPECS, ids=[s.name for s in SPECS])
@pytest.mark.parametrize("variant", ["fresh", "memo", "sthosvd"])
def test_bf16_tucker(ctx, spec, variant):
    import torch
    import paper_2507_23207_gb300 as K
    x, _, _ = tucker_tensor(spec)
    xb = philox.round_to_bf16(x)
    p = spec.oversample
    ells = [r + p for r in spec.ranks]
    memo, seq = variant == "memo", variant == "sthosvd"
    flags = (K.KRP_MEMO if memo else 0) | K.KRP_RESIDUAL
    core = torch.empty(int(np.prod(ells)), dtype=torch.float32, device=dev())
    facs = [torch.empty(n * l, dtype=torch.float64, device=dev()) for n, l in zip(spec.dims, ells)]
    fn = K.krp_tucker_sthosvd if seq else K.krp_tucker_rhosvd
    res = fn(ctx, tensor_to_dev(xb, torch.bfloat16), spec.dims, spec.ranks, p, 0, flags, core, facs)
    torch.cuda.synchronize()
    g = core.cpu().numpy().reshape(ells[::-1]).T.astype(np.float64)
    qs = [f.cpu().numpy().reshape(l, n).T for f, n, l in zip(facs, spec.dims, ells)]
    if seq:
        # step 1 sketches the BF16 X with BF16 factors; later steps FP32 cores
        ora = _sthosvd_bf16_first(xb, ells)
    else:
        ora = TK.rhosvd_krp(xb, ells, 0, memo=memo, omega_round="bf16")
    nx = np.linalg.norm(xb)
    for q in qs:
        assert np.linalg.norm(q.T @ q - np.eye(q.shape[1])) <= 1e-12
    xh = TK.reconstruct(g, qs)
    d2 = np.linalg.norm(xh - TK.reconstruct(ora["G"], ora["Q"])) / nx
    assert d2 <= 5e-5
    e_self = TK.rel_error(xb, g, qs)
    rho = eval_bound(ells, spec.dims, np.linalg.norm(xh) / nx, e_self, U_BF16_PAIR)
    check_error_value(res["rel_residual"], TK.rel_error(xb, ora["G"], ora["Q"]), e_self, d2, rho,
                      f"{spec.name}/{variant}")


def _sthosvd_bf16_first(x, ells):
    """Alg. 8 with the step-1 factors rounded to BF16 and later ones to FP32."""
    g = x
    qs, cores = [], [x]
    for i in range(x.ndim):
        om = TK.sthosvd_factors(0, g.shape, i, ells[i], omega_round="bf16" if i == 0 else "f32")
        y = T.mttkrp(g, om, i)
        q, _ = L.householder_qr(y)
        g = T.ttm(g, q.T, i)
        qs.append(q)
        cores.append(g)
    return {"G": g, "Q": qs}


def test_bf16_requires_aligned_first_mode(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    dims, ell = (37, 8, 8), 4
    x, om = bf16_case(dims, ell)
    y = empty_mat(37, ell, torch.float32)
    with pytest.raises(K.KrpError) as e:
        K.krp_sketch_mode(ctx, tensor_to_dev(x, torch.bfloat16), dims, 0,
                          [mat_to_dev(o, torch.bfloat16) for o in om], ell, y)
    assert e.value.status == K.KRP_EINVAL


# ---- BF16 hi/lo form (KRP_BF16X2): X streamed as two BF16 planes -------------

def _split_host(x):
    hi = philox.round_to_bf16(x)
    lo = philox.round_to_bf16(x - hi)
    return hi, lo


def _x2_dev(hi, lo):
    import torch
    import paper_2507_23207_gb300 as K
    h = tensor_to_dev(hi, torch.bfloat16).reshape(-1)
    l_ = tensor_to_dev(lo, torch.bfloat16).reshape(-1)
    return K.BF16x2(torch.cat([h, l_]))


def test_split_bf16x2_matches_host_split(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    rng = np.random.default_rng(11)
    x = philox.round_to_f32(rng.standard_normal(5003) * 10.0 ** rng.integers(-3, 3, 5003))
    xd = torch.from_numpy(x.astype(np.float32)).to(dev())
    x2 = K.krp_split_bf16x2(ctx, xd)
    torch.cuda.synchronize()
    got = x2.tensor.to(torch.float64).cpu().numpy()
    hi, lo = _split_host(x)
    assert np.array_equal(got[:5003], hi) and np.array_equal(got[5003:], lo)
    assert np.max(np.abs(hi + lo - x) / np.abs(x)) <= 2.0 ** -17


@pytest.mark.parametrize("dims,ell", [((64, 48, 40), 5), ((200, 200, 7), 30), ((256, 64, 16, 3), 12),
                                      ((136, 40, 30), 64), ((1024, 72, 5), 40), ((1024, 40, 6), 64)])
def test_bf16x2_sketches(ctx, dims, ell):
    """Sketch of hi + lo with BF16 factors: products exact, FP32 accumulation
    (all modes: the one-pass tree with the lo plane; mode 1 alone: the
    MTTKRP kernel)."""
    import torch
    import paper_2507_23207_gb300 as K
    rng = np.random.default_rng(sum(dims) + ell)
    x = philox.round_to_f32(np.asfortranarray(rng.standard_normal(dims)))
    hi, lo = _split_host(x)
    xe = hi + lo
    om = [philox.round_to_bf16(philox.gaussian_factor(9, j, 0, 0, n, ell)) for j, n in enumerate(dims)]
    x2 = _x2_dev(hi, lo)
    omd = [mat_to_dev(o, torch.bfloat16) for o in om]
    ys = [empty_mat(n, ell, torch.float32) for n in dims]
    K.krp_sketch_all_modes(ctx, x2, dims, omd, ell, ys)
    y0 = empty_mat(dims[0], ell, torch.float32)
    K.krp_sketch_mode(ctx, x2, dims, 0, omd, ell, y0)
    torch.cuda.synchronize()
    for n in range(len(dims)):
        assert rel(mat_from_dev(ys[n], dims[n], ell), T.mttkrp(xe, om, n)) <= 1e-5, (dims, n)
    assert rel(mat_from_dev(y0, dims[0], ell), T.mttkrp(xe, om, 0)) <= 1e-5


@pytest.mark.parametrize("variant", ["memo", "sthosvd"])
def test_bf16x2_tucker_truncated(ctx, variant):
    """RHOSVD-KRP-MEMO / RSTHOSVD-KRP with truncation on X = hi + lo against the
    oracle on hi + lo (BF16 factors): the core's MMAs drop only Xl Ql and
    Ql Hl-type terms (below 2^-16 relative)."""
    import torch
    import paper_2507_23207_gb300 as K
    spec = TuckerSpec("x2", (64, 48, 40), (4, 4, 4), 1e-3, None, 47, (4, 4, 4), (8, 8, 8))
    x, _, _ = tucker_tensor(spec)
    hi, lo = _split_host(philox.round_to_f32(x))
    xe = hi + lo
    p = spec.oversample
    ranks = list(spec.ranks)
    flags = K.KRP_TRUNCATE | K.KRP_RESIDUAL | (K.KRP_MEMO if variant == "memo" else 0)
    core = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device=dev())
    facs = [torch.empty(n * r, dtype=torch.float64, device=dev()) for n, r in zip(spec.dims, ranks)]
    fn = K.krp_tucker_rhosvd if variant == "memo" else K.krp_tucker_sthosvd
    res = fn(ctx, _x2_dev(hi, lo), spec.dims, ranks, p, 0, flags, core, facs)
    torch.cuda.synchronize()
    ells = [r + p for r in ranks]
    if variant == "memo":
        ora = TK.rhosvd_krp(xe, ells, 0, memo=True, omega_round="bf16")
    else:
        ora = _sthosvd_bf16_first(xe, ells)
    g2, q2 = TK.truncate_core(ora["G"], ora["Q"], ranks)
    gg = core.cpu().numpy().astype(np.float64).reshape(ranks[::-1]).T
    qq = [f.cpu().numpy().reshape(r, n).T for f, n, r in zip(facs, spec.dims, ranks)]
    nx = np.linalg.norm(xe)
    xh = TK.reconstruct(gg, qq)
    d2 = np.linalg.norm(xh - TK.reconstruct(g2, q2)) / nx
    assert d2 <= 5e-5
    e_self = TK.rel_error(xe, gg, qq)
    rho = eval_bound(ranks, spec.dims, np.linalg.norm(xh) / nx, e_self, U_BF16_PAIR)
    check_error_value(res["rel_residual"], TK.rel_error(xe, g2, q2), e_self, d2, rho, variant)
