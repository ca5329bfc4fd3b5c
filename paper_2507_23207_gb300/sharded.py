"""RHOSVD-KRP-MEMO of one tensor sharded across ranks (one GPU each).

X is split into contiguous slabs of its last (slowest) mode, one per rank.
Each rank computes only slab-local partial results, and the ranks exchange
small sums (an all-reduce):

1. every rank draws the same factor set {Omega_j} (the Philox stream is
   counter-based, Sec. 2.5), and keeps the rows [start, stop) of Omega_d;
2. sketches of the slab (Alg. 7, memoized, one pass over the slab): for
   n < d the slab's Y_n is a partial sum of the full Y_n (the slabs partition
   the rows of the Khatri-Rao product); for n = d it is the block of rows
   [start, stop) of Y_d.  One all-reduce of sum_n n_n l values, all d
   sketches packed into one buffer (Y_d padded with zeros outside the slab's
   rows);
3. the FP64 QR of every Y_n runs on every rank (replicated, identical);
4. core G = X x {Q_n^T}: with Q_d's rows [start, stop) the slab gives a
   partial sum of G; one all-reduce of prod_n l_n values;
5. truncation of the core (replicated) and the residual sums of the slab
   (||X_s - X_hat_s||^2, ||X_s||^2 with the slab's rows of the last factor),
   one all-reduce of two values.

The per-rank steps go through an ``ops`` object; ``CudaOps`` runs them in
the CUDA library through the C ABI.  All arrays are flat tensors in the C
ABI's layouts: X and cores mode-1 fastest, factors, sketches and Q's
column-major n x l.  The exchange is ``torch.distributed.all_reduce`` (NCCL
for CUDA tensors) unless another reducer is passed.
"""

from __future__ import annotations

import math
from typing import Callable, List, Optional, Sequence, Tuple

import torch

from . import krp as K


def slab_bounds(n_last: int, world: int, rank: int) -> Tuple[int, int]:
    """Rows [start, stop) of the last mode owned by `rank`: contiguous slabs,
    sizes differing by at most one."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} out of range for world {world}")
    if n_last < world:
        raise ValueError(f"last mode ({n_last}) has fewer slabs than ranks ({world})")
    base, extra = divmod(n_last, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def rows_of(mat: torch.Tensor, n: int, ell: int, start: int, stop: int) -> torch.Tensor:
    """Rows [start, stop) of a flat column-major n x ell matrix, flat column-major."""
    return mat.view(ell, n)[:, start:stop].contiguous().view(-1)


def place_rows(full: torch.Tensor, block: torch.Tensor, n: int, ell: int, start: int, stop: int):
    """full (flat column-major n x ell)[start:stop, :] = block (flat column-major)."""
    full.view(ell, n)[:, start:stop] = block.view(ell, stop - start)


class CudaOps:
    """Per-rank steps through the C ABI, on the context's GPU."""

    def __init__(self, ctx: K.Context, device):
        self.ctx = ctx
        self.device = torch.device(device)

    def factors(self, seed: int, dims: Sequence[int], ell: int, dtype) -> List[torch.Tensor]:
        om = [torch.empty(n * ell, dtype=dtype, device=self.device) for n in dims]
        K.krp_gen_factors(self.ctx, seed, K.KRP_DRAW_MEMO, K.KRP_TAG_OMEGA, dims, ell, om)
        return om

    def sketch_all(self, x, dims: Sequence[int], omegas: Sequence[torch.Tensor], ell: int):
        ys = [torch.empty(n * ell, dtype=torch.float32, device=self.device) for n in dims]
        K.krp_sketch_all_modes(self.ctx, x, dims, omegas, ell, ys)
        return ys

    def qr(self, ys: Sequence[torch.Tensor], dims: Sequence[int], ells: Sequence[int]):
        qs = [torch.empty(n * l, dtype=torch.float64, device=self.device)
              for n, l in zip(dims, ells)]
        K.krp_qr(self.ctx, ys, dims, ells, qs)
        return qs

    def multi_ttm(self, x, dims: Sequence[int], qs: Sequence[torch.Tensor], cols: Sequence[int]):
        g = torch.empty(math.prod(cols), dtype=torch.float32, device=self.device)
        K.krp_multi_ttm(self.ctx, x, dims, qs, cols, g)
        return g

    def truncate(self, dims, ells, ranks, core, qs):
        g = torch.empty(math.prod(ranks), dtype=torch.float32, device=self.device)
        qr_ = [torch.empty(n * r, dtype=torch.float64, device=self.device)
               for n, r in zip(dims, ranks)]
        K.krp_core_truncate(self.ctx, dims, ells, ranks, core, qs, g, qr_)
        return g, qr_

    def residual(self, x, dims, core_dims, core, qs) -> Tuple[float, float]:
        return K.krp_residual(self.ctx, x, dims, core_dims, core, qs)


def _dist_allreduce(t: torch.Tensor) -> None:
    import torch.distributed as dist
    dist.all_reduce(t)


def exchange_bytes(dims: Sequence[int], ranks: Sequence[int], oversample: int,
                   residual: bool = True) -> int:
    """Bytes each rank contributes to the all-reduces of one sharded call:
    the packed sketches (sum_n n_n l, FP32), the core (prod l_n, FP32) and the
    two residual sums (FP64)."""
    ells = [int(r) + oversample for r in ranks]
    return 4 * sum(int(n) * max(ells) for n in dims) + 4 * math.prod(ells) + (16 if residual else 0)


def rhosvd_sharded(ops, x_local, dims: Sequence[int], start: int, stop: int,
                   ranks: Sequence[int], oversample: int, seed: int, *,
                   truncate: bool = True, residual: bool = True,
                   factor_dtype=torch.float32,
                   allreduce: Optional[Callable[[torch.Tensor], None]] = None):
    """RHOSVD-KRP-MEMO of the whole tensor from this rank's slab X[..., start:stop].

    Returns (core, factors, rel_residual or None): core flat FP32 of the
    ranks (or ell_n = ranks[n] + oversample without truncation), factors flat
    FP64 n_n x rank_n, identical on every rank.
    """
    reduce = allreduce or _dist_allreduce
    d = len(dims)
    dims = [int(n) for n in dims]
    ells = [int(r) + oversample for r in ranks]
    ellmax = max(ells)
    local = dims[:-1] + [stop - start]
    if stop <= start:
        raise ValueError("empty slab")
    omegas = ops.factors(seed, dims, ellmax, factor_dtype)
    om_local = list(omegas[:-1]) + [rows_of(omegas[-1], dims[-1], ellmax, start, stop)]
    ys = ops.sketch_all(x_local, local, om_local, ellmax)
    yd = torch.zeros(dims[-1] * ellmax, dtype=ys[-1].dtype, device=ys[-1].device)
    place_rows(yd, ys[-1], dims[-1], ellmax, start, stop)
    ys[-1] = yd
    # one exchange for all d sketches: partial sums (n < d) and disjoint row
    # blocks (n = d) packed into one buffer
    sizes = [y.numel() for y in ys]
    packed = torch.cat(ys)
    reduce(packed)
    ys = list(torch.split(packed, sizes))
    qs = ops.qr([y[: n * l] for y, n, l in zip(ys, dims, ells)], dims, ells)
    q_local = list(qs[:-1]) + [rows_of(qs[-1], dims[-1], ells[-1], start, stop)]
    core = ops.multi_ttm(x_local, local, q_local, ells)
    reduce(core)
    cdims = ells
    if truncate:
        core, qs = ops.truncate(dims, ells, list(ranks), core, qs)
        cdims = list(ranks)
    rel = None
    if residual:
        q_local = list(qs[:-1]) + [rows_of(qs[-1], dims[-1], cdims[-1], start, stop)]
        d2, x2 = ops.residual(x_local, local, cdims, core, q_local)
        sums = torch.tensor([d2, x2], dtype=torch.float64, device=core.device)
        reduce(sums)
        rel = math.sqrt(float(sums[0]) / float(sums[1])) if float(sums[1]) > 0 else 0.0
    return core, qs, rel
