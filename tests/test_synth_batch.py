"""The seeded batched workloads: 512 uneven tensors and 64 block Hankel
matrices with the shapes, ranks and keys the batched entry points are
benchmarked on (sides U(32..192), ranks U(4..16), l = r + 8; Hankel order
U(8..32) even, m = n U(4..8), s U(32..128), l_r = r + 8, l_l = ceil(1.5 l_r)).
Every item is valid for the batched C ABI (l_i <= min(32, n_i); l_r <= 64,
l_l <= 256), and the batch is reproducible."""

import math

from synth import batch_hankel_specs, batch_tucker_specs


def test_tucker_batch_shapes_ranks_and_keys():
    specs = batch_tucker_specs(512)
    assert len(specs) == 512
    sides = [n for sp in specs for n in sp.dims]
    ranks = [r for sp in specs for r in sp.ranks]
    assert min(sides) >= 32 and max(sides) <= 192
    assert min(ranks) >= 4 and max(ranks) <= 16
    # the draws cover their ranges (512 x 3 draws of 161 and 13 values)
    assert min(sides) <= 35 and max(sides) >= 189 and len(set(ranks)) == 13
    for b, sp in enumerate(specs):
        assert sp.ell == tuple(r + 8 for r in sp.ranks)
        assert all(l <= min(32, n) for l, n in zip(sp.ell, sp.dims))
        assert sp.omega_seed == b
    assert [sp.data_seed for sp in specs] == [1005 + b for b in range(512)]
    again = batch_tucker_specs(512)
    assert [(s.dims, s.ranks, s.data_seed) for s in again] == \
        [(s.dims, s.ranks, s.data_seed) for s in specs]
    # about 7.3e8 entries in total (E[n]^3 = 112^3 ~ 1.4e6 per tensor)
    total = sum(math.prod(sp.dims) for sp in specs)
    assert 5e8 < total < 1e9


def test_hankel_batch_orders_blocks_and_sketch_sizes():
    specs = batch_hankel_specs(64)
    assert len(specs) == 64
    for b, sp in enumerate(specs):
        assert 8 <= sp.order <= 32 and sp.order % 2 == 0
        assert 4 <= sp.m <= 8 and sp.n == sp.m
        assert 32 <= sp.s <= 128
        assert sp.r == sp.order and sp.ell_r == sp.order + 8
        assert sp.ell_l == math.ceil(1.5 * sp.ell_r)
        assert sp.ell_r <= 64 and sp.ell_l <= 256
        assert sp.ell_r <= sp.m * sp.s and sp.ell_l <= sp.n * sp.s
        assert sp.omega_seed == b
