"""Sharded RHOSVD-KRP-MEMO (one slab of the last mode per rank): the
orchestration of paper_2507_23207_gb300.sharded run on two CPU ranks (gloo
all-reduce over 127.0.0.1), with the per-rank steps taken by the FP64 oracle
(a test backend; the product backend is CudaOps).  The sharded result must be
the unsharded oracle pipeline's (Alg. 7 with the memoized factor set, then the
HOSVD truncation of the core and the residual) up to FP64 rounding; without
the exchange it must not be.
"""

import math
import os
import socket

import numpy as np
import pytest
import torch

from oracle import linalg as L
from oracle import philox
from oracle import tensor as T
from oracle import tucker as TK
from paper_2507_23207_gb300.sharded import place_rows, rhosvd_sharded, rows_of, slab_bounds


def _flat(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.asarray(a, dtype=np.float64).flatten(order="F").copy())


def _arr(t: torch.Tensor, shape) -> np.ndarray:
    return t.numpy().reshape(shape, order="F")


class OracleOps:
    """The per-rank steps in FP64 by the oracle, on flat CPU tensors."""

    def factors(self, seed, dims, ell, dtype):
        return [_flat(f) for f in philox.krp_factors(seed, TK.MEMO_DRAW, dims, ell)]

    def sketch_all(self, x, dims, omegas, ell):
        xa = _arr(x, dims)
        oms = [_arr(o, (n, ell)) for o, n in zip(omegas, dims)]
        return [_flat(T.mttkrp(xa, oms, n)) for n in range(len(dims))]

    def qr(self, ys, dims, ells):
        return [_flat(L.householder_qr(_arr(y, (n, l)))[0]) for y, n, l in zip(ys, dims, ells)]

    def multi_ttm(self, x, dims, qs, cols):
        qa = [_arr(q, (n, c)) for q, n, c in zip(qs, dims, cols)]
        return _flat(T.multi_ttm(_arr(x, dims), [q.T for q in qa]))

    def truncate(self, dims, ells, ranks, core, qs):
        g, q2 = TK.truncate_core(_arr(core, ells), [_arr(q, (n, l)) for q, n, l in
                                                     zip(qs, dims, ells)], ranks)
        return _flat(g), [_flat(q) for q in q2]

    def residual(self, x, dims, core_dims, core, qs):
        xa = _arr(x, dims)
        qa = [_arr(q, (n, c)) for q, n, c in zip(qs, dims, core_dims)]
        r = xa - TK.reconstruct(_arr(core, core_dims), qa)
        return float(np.sum(r * r)), float(np.sum(xa * xa))


CASES = [((9, 8, 7), (3, 3, 2), 2), ((6, 5, 4, 5), (2, 2, 2, 2), 1)]


def _tensor(dims, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(dims)


def _expected(x, ranks, oversample, seed):
    ells = [r + oversample for r in ranks]
    ora = TK.rhosvd_krp(x, ells, seed, memo=True)
    g, qs = TK.truncate_core(ora["G"], ora["Q"], ranks)
    return g, qs, TK.rel_error(x, g, qs)


def _rank_main(rank, world, port, case_idx):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims, ranks, p = CASES[case_idx]
        seed = 5
        x = _tensor(dims, 100 + case_idx)
        start, stop = slab_bounds(dims[-1], world, rank)
        x_local = _flat(x[..., start:stop])
        core, qs, rel = rhosvd_sharded(OracleOps(), x_local, dims, start, stop, ranks, p, seed)
        g_exp, q_exp, rel_exp = _expected(x, ranks, p, seed)
        qa = [_arr(q, (n, r)) for q, n, r in zip(qs, dims, ranks)]
        xh = TK.reconstruct(_arr(core, ranks), qa)
        xh_exp = TK.reconstruct(g_exp, q_exp)
        nx = np.linalg.norm(x)
        assert np.linalg.norm(xh - xh_exp) <= 1e-12 * nx, (rank, np.linalg.norm(xh - xh_exp) / nx)
        assert abs(rel - rel_exp) <= 1e-12, (rank, rel, rel_exp)
        for q in qa:
            assert np.linalg.norm(q.T @ q - np.eye(q.shape[1])) <= 1e-12
        # the exchange matters: without it each rank sees only its slab
        core0, qs0, rel0 = rhosvd_sharded(OracleOps(), x_local, dims, start, stop, ranks, p, seed,
                                          allreduce=lambda t: None)
        qa0 = [_arr(q, (n, r)) for q, n, r in zip(qs0, dims, ranks)]
        xh0 = TK.reconstruct(_arr(core0, ranks), qa0)
        assert np.linalg.norm(xh0 - xh_exp) > 1e-3 * nx
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("case_idx", range(len(CASES)))
def test_sharded_two_gloo_ranks_match_unsharded_oracle(case_idx):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), case_idx), nprocs=2, join=True)


@pytest.mark.parametrize("world,case_idx", [(3, 0), (4, 1)])
def test_sharded_more_ranks_than_two_uneven_slabs(world, case_idx):
    # 7 slabs over 3 ranks and 5 slabs over 4 ranks: unequal slab counts per rank
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, _free_port(), case_idx), nprocs=world, join=True)


def test_single_rank_is_the_unsharded_pipeline():
    dims, ranks, p = CASES[0]
    x = _tensor(dims, 7)
    core, qs, rel = rhosvd_sharded(OracleOps(), _flat(x), dims, 0, dims[-1], ranks, p, 3,
                                   allreduce=lambda t: None)
    g_exp, q_exp, rel_exp = _expected(x, ranks, p, 3)
    qa = [_arr(q, (n, r)) for q, n, r in zip(qs, dims, ranks)]
    assert np.linalg.norm(TK.reconstruct(_arr(core, ranks), qa) - TK.reconstruct(g_exp, q_exp)) \
        <= 1e-12 * np.linalg.norm(x)
    assert abs(rel - rel_exp) <= 1e-12


def test_slab_bounds_partition_the_last_mode():
    for n in (7, 8, 100, 1024):
        for world in (1, 2, 3, 7):
            if n < world:
                continue
            spans = [slab_bounds(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slab_bounds(3, 4, 0)


def test_row_slicing_helpers():
    n, ell = 7, 3
    m = torch.arange(n * ell, dtype=torch.float64)  # column-major n x ell
    blk = rows_of(m, n, ell, 2, 5)
    a = m.numpy().reshape((n, ell), order="F")
    assert np.array_equal(blk.numpy().reshape((3, ell), order="F"), a[2:5])
    full = torch.zeros(n * ell, dtype=torch.float64)
    place_rows(full, blk, n, ell, 2, 5)
    fa = full.numpy().reshape((n, ell), order="F")
    assert np.array_equal(fa[2:5], a[2:5]) and not fa[:2].any() and not fa[5:].any()


def test_one_exchange_per_phase():
    """The d sketches travel in one packed all-reduce: a call makes exactly
    three exchanges (sketches, core, residual sums) carrying
    exchange_bytes() bytes, whatever d is."""
    from paper_2507_23207_gb300.sharded import exchange_bytes
    for dims, ranks in (((9, 8, 7), (2, 2, 2)), ((6, 5, 4, 5), (2, 2, 2, 2))):
        rng = np.random.default_rng(5)
        x = rng.standard_normal(dims)
        calls = []

        def count(t):
            calls.append(t.numel() * t.element_size())
        core, qs, rel = rhosvd_sharded(OracleOps(), _flat(x), dims, 0, dims[-1], ranks, 2, 0,
                                       allreduce=count, factor_dtype=torch.float64)
        assert len(calls) == 3, calls
        # FP64 buffers here; the CUDA path exchanges FP32 sketches and core
        assert sum(calls) == 2 * (exchange_bytes(dims, ranks, 2) - 16) + 16
