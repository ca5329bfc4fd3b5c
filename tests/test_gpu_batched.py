"""a11: the batched uneven Tucker path against the FP64 oracle, per tensor.

Each tensor b of a batch is RHOSVD-KRP-MEMO with its own Philox key seed_b, so
the oracle's rhosvd_krp(X_b, l, seed_b, memo=True) (+ truncation) is the
reference: FP32 form within 1e-5 (reconstruction relative to ||X_b||); error
values within 1e-5 relative, widened by the measured reconstruction distance
and the residual pass's rounding bound (tests/parity.py; the factors enter
the FP32 reconstruction rounded, Q~_i = Q_i + E_i).  BF16 form (X and factors rounded to BF16, FP32 arithmetic
on CUDA cores): the same bounds on the BF16-rounded data.  Also: a repeated call
replays the captured graph with identical results, and new descriptors build
a new plan.
"""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, tensor_to_dev
from tests.parity import check_error_value, eval_bound
from oracle import philox, tucker as TK
from synth import TuckerSpec, tucker_tensor

pytestmark = pytest.mark.gpu

P = 4
SHAPES = [((40, 33, 27), (3, 4, 2)), ((5, 7, 9), (1, 2, 2)), ((64, 16, 48), (6, 5, 8)),
          ((31, 90, 12), (4, 4, 4)), ((96, 40, 70), (8, 3, 6)), ((17, 17, 17), (2, 2, 3)),
          ((128, 50, 33), (12, 9, 16)), ((8, 200, 24), (4, 16, 10)),
          # l up to 32: the widest kernel variants (8 n-tiles of the warp MMAs,
          # 32 accumulators per lane on CUDA cores)
          ((48, 40, 36), (24, 26, 28))]


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


def _batch(dtype, flags_trunc, shapes=SHAPES, seed0=500):
    import torch
    xs, hosts, dims, ranks, seeds, cores, facs = [], [], [], [], [], [], []
    for b, (d, r) in enumerate(shapes):
        spec = TuckerSpec(f"t{b}", d, tuple(min(n, rr + 2) for n, rr in zip(d, r)), 1e-3, None,
                          77 + b, r, tuple(rr + P for rr in r))
        x, _, _ = tucker_tensor(spec)
        x = philox.round_to_bf16(x) if dtype == torch.bfloat16 else philox.round_to_f32(x)
        hosts.append(x)
        xs.append(tensor_to_dev(x, dtype))
        dims.append(d)
        ranks.append(r)
        seeds.append(seed0 + b)
        out = r if flags_trunc else tuple(rr + P for rr in r)
        cores.append(torch.empty(int(np.prod(out)), dtype=torch.float32, device=dev()))
        facs.append([torch.empty(n * o, dtype=torch.float64, device=dev()) for n, o in zip(d, out)])
    return xs, hosts, dims, ranks, seeds, cores, facs


def _check(hosts, ranks, seeds, cores, facs, rels, trunc, omega_round, tol):
    for b, x in enumerate(hosts):
        ells = [r + P for r in ranks[b]]
        ora = TK.rhosvd_krp(x, ells, seeds[b], memo=True, omega_round=omega_round)
        g, qs = ora["G"], ora["Q"]
        if trunc:
            g, qs = TK.truncate_core(g, qs, list(ranks[b]))
        out = list(ranks[b]) if trunc else ells
        gg = cores[b].cpu().numpy().astype(np.float64).reshape(out[::-1]).T
        qq = [f.cpu().numpy().reshape(o, n).T for f, n, o in zip(facs[b], x.shape, out)]
        nx = np.linalg.norm(x)
        xh = TK.reconstruct(gg, qq)
        d = np.linalg.norm(xh - TK.reconstruct(g, qs)) / nx
        assert d <= tol, (b, x.shape, d)
        e_ora = TK.rel_error(x, g, qs)
        e_self = TK.rel_error(x, gg, qq)
        rho = eval_bound(out, x.shape, np.linalg.norm(xh) / nx, e_self)
        check_error_value(rels[b], e_ora, e_self, d, rho, f"item {b} {x.shape}")
        for q in qq:
            assert np.linalg.norm(q.T @ q - np.eye(q.shape[1])) <= 1e-10


@pytest.mark.parametrize("form", ["f32", "bf16"])
@pytest.mark.parametrize("trunc", [True, False])
def test_batched_matches_oracle(ctx, form, trunc):
    import torch
    import paper_2507_23207_gb300 as K
    dtype = torch.float32 if form == "f32" else torch.bfloat16
    xs, hosts, dims, ranks, seeds, cores, facs = _batch(dtype, trunc)
    items = K.make_tucker_items(xs, dims, ranks, seeds, cores, facs)
    flags = (K.KRP_TRUNCATE if trunc else 0) | K.KRP_RESIDUAL
    rels = K.krp_tucker_rhosvd_batched(ctx, K.KRP_F32 if form == "f32" else K.KRP_BF16, items, P,
                                       flags)
    torch.cuda.synchronize()
    _check(hosts, ranks, seeds, cores, facs, rels, trunc, form, 1e-5)


# sides at the limit (256: one 32-column panel of pitch 264 per copy in the
# staged BF16 sketch), odd sides, and several panels per slab
EDGE_SHAPES = [((256, 20, 9), (4, 3, 2)), ((7, 256, 6), (2, 6, 2)), ((33, 65, 7), (3, 3, 2)),
               ((200, 190, 6), (5, 5, 2)), ((9, 250, 11), (3, 7, 4))]


@pytest.mark.parametrize("aligned", [True, False])
def test_batched_bf16_edge_shapes(ctx, aligned):
    """BF16 batch at the side limit and with odd sides; aligned=False packs all
    tensors into one buffer at odd element offsets, so no tensor starts or ends
    on a 16-byte boundary (the staged sketch copies the aligned interior of
    each panel and reads the ends with plain loads)."""
    import torch
    import paper_2507_23207_gb300 as K
    xs, hosts, dims, ranks, seeds, cores, facs = _batch(torch.bfloat16, True, EDGE_SHAPES, 700)
    if not aligned:
        sizes = [x.numel() for x in xs]
        buf = torch.empty(sum(sizes) + 3 * len(xs) + 1, dtype=torch.bfloat16, device=dev())
        views, off = [], 1
        for x, n in zip(xs, sizes):
            v = buf[off:off + n]
            v.copy_(x.reshape(-1))
            views.append(v)
            assert (v.data_ptr() % 16) != 0
            off += n + 2
            off += 1 if off % 8 == 0 else 0
        xs = views
    items = K.make_tucker_items(xs, dims, ranks, seeds, cores, facs)
    rels = K.krp_tucker_rhosvd_batched(ctx, K.KRP_BF16, items, P, K.KRP_TRUNCATE | K.KRP_RESIDUAL)
    torch.cuda.synchronize()
    _check(hosts, ranks, seeds, cores, facs, rels, True, "bf16", 1e-5)


def test_batched_graph_replay_and_rebuild(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    xs, hosts, dims, ranks, seeds, cores, facs = _batch(torch.float32, True)
    items = K.make_tucker_items(xs, dims, ranks, seeds, cores, facs)
    flags = K.KRP_TRUNCATE | K.KRP_RESIDUAL
    r1 = K.krp_tucker_rhosvd_batched(ctx, K.KRP_F32, items, P, flags)
    info = K.krp_tucker_batch_plan_info(ctx)
    assert info["slabs_per_unit"] in (2, 4, 8, 16) and info["units"] >= len(SHAPES)
    def recon(b):
        out = list(ranks[b])
        g = cores[b].cpu().numpy().astype(np.float64).reshape(out[::-1]).T
        qs = [f.cpu().numpy().reshape(o, n).T for f, n, o in zip(facs[b], dims[b], out)]
        return TK.reconstruct(g, qs)

    x1 = [recon(b) for b in range(len(SHAPES))]
    for c in cores:
        c.zero_()
    r2 = K.krp_tucker_rhosvd_batched(ctx, K.KRP_F32, items, P, flags)
    assert K.krp_tucker_batch_plan_info(ctx) == info
    # the replay recomputes everything (cores were cleared); atomics may sum in
    # another order, so compare basis-invariant results
    for b in range(len(SHAPES)):
        assert np.linalg.norm(recon(b) - x1[b]) <= 1e-5 * np.linalg.norm(hosts[b])
    assert np.allclose(r1, r2, rtol=1e-4)
    # other seeds: a new plan, results follow the oracle for the new seeds
    seeds2 = [s + 1000 for s in seeds]
    items2 = K.make_tucker_items(xs, dims, ranks, seeds2, cores, facs)
    rels = K.krp_tucker_rhosvd_batched(ctx, K.KRP_F32, items2, P, flags)
    _check(hosts, ranks, seeds2, cores, facs, rels, True, "f32", 1e-5)


def test_batched_rejects_bad_descriptors(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    xs, hosts, dims, ranks, seeds, cores, facs = _batch(torch.float32, True, SHAPES[:2])
    bad = [list(r) for r in ranks]
    bad[1][0] = dims[1][0]  # l = r + P > n
    items = K.make_tucker_items(xs, dims, bad, seeds, cores, facs)
    with pytest.raises(K.KrpError) as e:
        K.krp_tucker_rhosvd_batched(ctx, K.KRP_F32, items, P, K.KRP_TRUNCATE)
    assert e.value.status == K.KRP_EINVAL


HSPECS = [(6, 3, 2, 9, 6, 10, 15), (10, 5, 3, 17, 10, 13, 20), (12, 8, 8, 40, 12, 20, 30),
          (8, 4, 4, 33, 8, 16, 24), (20, 6, 6, 64, 20, 28, 42)]


def _hankel_batch(dtype):
    import torch
    from synth import HankelSpec, markov_parameters
    blocks, hosts, shapes, seeds, Us, Ss, Vs = [], [], [], [], [], [], []
    for b, (order, m, n, s, r, lr, ll) in enumerate(HSPECS):
        spec = HankelSpec(f"h{b}", order, m, n, s, 0.9, 300 + b, r, lr, ll)
        bl = markov_parameters(spec)
        bl = philox.round_to_bf16(bl) if dtype == torch.bfloat16 else philox.round_to_f32(bl)
        hosts.append(bl)
        flat = np.concatenate([np.asfortranarray(bl[:, :, k]).ravel(order="F")
                               for k in range(bl.shape[2])])
        blocks.append(torch.from_numpy(flat).to(dtype).to(dev()))
        shapes.append((m, n, s, r, lr, ll))
        seeds.append(40 + b)
        Us.append(torch.empty((r, m * s), dtype=torch.float64, device=dev()))
        Vs.append(torch.empty((r, n * s), dtype=torch.float64, device=dev()))
        Ss.append(torch.empty(r, dtype=torch.float64, device=dev()))
    return blocks, hosts, shapes, seeds, Us, Ss, Vs


@pytest.mark.parametrize("form", ["f32", "bf16"])
def test_batched_hankel_matches_oracle(ctx, form):
    """Every matrix of the batch against the oracle's Alg. 6 with the same key:
    singular values (relative to sigma_1) and U S V^T (relative to ||H||)."""
    import torch
    import paper_2507_23207_gb300 as K
    from oracle import hankel as HK
    dtype = torch.float32 if form == "f32" else torch.bfloat16
    blocks, hosts, shapes, seeds, Us, Ss, Vs = _hankel_batch(dtype)
    items = K.make_hankel_items(blocks, shapes, seeds, Us, Ss, Vs)
    for rep in range(2):  # first call builds and captures, second replays
        for u in Us:
            u.zero_()
        K.krp_block_hankel_batched(ctx, K.KRP_F32 if form == "f32" else K.KRP_BF16, items)
        torch.cuda.synchronize()
        for b, bl in enumerate(hosts):
            m, n, s, r, lr, ll = shapes[b]
            ora = HK.single_pass_svd(bl, r, lr, ll, seeds[b], omega_round=form)
            ug = Us[b].cpu().numpy().T
            vg = Vs[b].cpu().numpy().T
            sg = Ss[b].cpu().numpy()
            assert np.max(np.abs(sg - ora["S"])) <= 1e-5 * ora["S"][0], (b, rep)
            ag = (ug * sg) @ vg.T
            ao = (ora["U"] * ora["S"]) @ ora["V"].T
            assert np.linalg.norm(ag - ao) <= 1e-5 * np.linalg.norm(ora["H"]), (b, rep)
