"""Sharded RHOSVD-KRP-MEMO through the C ABI (CudaOps), and the two entry
points it adds, krp_core_truncate and krp_residual.

Two ranks are emulated by two host threads on one GPU, each with its own
context and slab of the last mode; the exchange is a host-side sum after
each thread has synchronised its stream (no kernel waits on another).  The
result must be the single-GPU pipeline's (krp_tucker_rhosvd with
KRP_MEMO | KRP_TRUNCATE | KRP_RESIDUAL) up to FP32 summation order.
"""

import math
import threading

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, tensor_to_dev
from tests.parity import U_F32, U_TF32_PAIR, check_error_value, eval_bound
from oracle import philox, tucker as TK
from synth import TuckerSpec, tucker_tensor

pytestmark = pytest.mark.gpu

SPECS = [
    TuckerSpec("s3", (64, 48, 40), (4, 4, 4), 1e-3, None, 61, (4, 4, 4), (8, 8, 8)),
    TuckerSpec("s4", (24, 20, 16, 18), (3, 3, 3, 3), 1e-3, None, 62, (3, 3, 3, 3), (6, 6, 6, 6)),
]


class ThreadReducer:
    """Sum across `n` threads of one process (each waits for the others)."""

    def __init__(self, n):
        self.n = n
        self.barrier = threading.Barrier(n)
        self.slots = [None] * n
        self.total = None

    def for_rank(self, r):
        def reduce(t):
            import torch
            torch.cuda.synchronize()
            self.slots[r] = t.clone()
            self.barrier.wait()
            if r == 0:
                total = self.slots[0].clone()
                for s in self.slots[1:]:
                    total += s
                self.total = total
            self.barrier.wait()
            t.copy_(self.total)
            torch.cuda.synchronize()
            self.barrier.wait()
        return reduce


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


def _single_gpu(ctx, xd, spec, flags):
    import torch
    import paper_2507_23207_gb300 as K
    ranks, p = list(spec.ranks), spec.oversample
    out = ranks if flags & K.KRP_TRUNCATE else [r + p for r in ranks]
    core = torch.empty(math.prod(out), dtype=torch.float32, device=dev())
    facs = [torch.empty(n * o, dtype=torch.float64, device=dev()) for n, o in zip(spec.dims, out)]
    res = K.krp_tucker_rhosvd(ctx, xd, spec.dims, ranks, p, 0, flags, core, facs)
    torch.cuda.synchronize()
    return core, facs, res


def _gq(core, facs, dims, cdims):
    g = core.cpu().numpy().astype(np.float64).reshape(cdims[::-1]).T
    qs = [f.cpu().numpy().reshape(c, n).T for f, n, c in zip(facs, dims, cdims)]
    return g, qs


def _recon(core, facs, dims, cdims):
    return TK.reconstruct(*_gq(core, facs, dims, cdims))


def _rho(x, core, facs, dims, cdims):
    """Exact error of a returned (core, factors) and the residual pass's
    rounding bound for it (tests/parity.py)."""
    g, qs = _gq(core, facs, dims, cdims)
    nx = np.linalg.norm(x)
    e_self = TK.rel_error(x, g, qs)
    return e_self, eval_bound(cdims, dims, np.linalg.norm(TK.reconstruct(g, qs)) / nx, e_self,
                              U_F32, U_TF32_PAIR)


@pytest.mark.parametrize("spec", SPECS, ids=[s.name for s in SPECS])
def test_core_truncate_and_residual_entry_points(ctx, spec):
    import torch
    import paper_2507_23207_gb300 as K
    x, _, _ = tucker_tensor(spec)
    x32 = philox.round_to_f32(x)
    xd = tensor_to_dev(x32, torch.float32)
    ranks, p = list(spec.ranks), spec.oversample
    ells = [r + p for r in ranks]
    core_l, facs_l, _ = _single_gpu(ctx, xd, spec, K.KRP_MEMO)
    core_t, facs_t, res_t = _single_gpu(ctx, xd, spec, K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL)
    # the entry point truncates the rank-l result as the pipeline does
    core_r = torch.empty(math.prod(ranks), dtype=torch.float32, device=dev())
    facs_r = [torch.empty(n * r, dtype=torch.float64, device=dev()) for n, r in zip(spec.dims, ranks)]
    K.krp_core_truncate(ctx, spec.dims, ells, ranks, core_l, facs_l, core_r, facs_r)
    torch.cuda.synchronize()
    nx = np.linalg.norm(x32)
    xr = _recon(core_r, facs_r, spec.dims, ranks)
    assert np.linalg.norm(xr - _recon(core_t, facs_t, spec.dims, ranks)) <= 1e-6 * nx
    for f, n, r in zip(facs_r, spec.dims, ranks):
        q = f.cpu().numpy().reshape(r, n).T
        assert np.linalg.norm(q.T @ q - np.eye(r)) <= 1e-12
    # ... and equals the oracle's truncation of the oracle's rank-l result
    ora = TK.rhosvd_krp(x32, ells, 0, memo=True, omega_round="f32")
    g_o, q_o = TK.truncate_core(ora["G"], ora["Q"], ranks)
    assert np.linalg.norm(xr - TK.reconstruct(g_o, q_o)) <= 1e-5 * nx
    # residual sums of the truncated approximation
    d2, x2 = K.krp_residual(ctx, xd, spec.dims, ranks, core_r, facs_r)
    # ||X||^2: FP32 partial sums of at most 64 squares per thread, then FP64
    assert abs(x2 - float(np.sum(x32.astype(np.float64) ** 2))) <= 64 * 2.0 ** -24 * x2
    # P3 against the oracle (tests/parity.py): 1e-5 relative, widened by the
    # measured reconstruction distance and the residual pass's rounding bound
    e_r = math.sqrt(d2 / x2)
    e_self, rho = _rho(x32, core_r, facs_r, spec.dims, ranks)
    eta_o = np.linalg.norm(xr - TK.reconstruct(g_o, q_o)) / nx
    check_error_value(e_r, TK.rel_error(x32, g_o, q_o), e_self, eta_o, rho, spec.name)
    # against the pipeline's own residual pass on its (slightly different:
    # FP32 atomics order) result: both within rho of their exact errors,
    # which differ by at most the reconstructions' distance
    eta_t = np.linalg.norm(xr - _recon(core_t, facs_t, spec.dims, ranks)) / nx
    e_self_t, rho_t = _rho(x32, core_t, facs_t, spec.dims, ranks)
    check_error_value(res_t["rel_residual"], e_r, e_self_t, eta_t, rho_t + rho, spec.name)


@pytest.mark.parametrize("spec", SPECS, ids=[s.name for s in SPECS])
def test_two_virtual_ranks_match_single_gpu_pipeline(ctx, spec):
    import torch
    import paper_2507_23207_gb300 as K
    from paper_2507_23207_gb300.sharded import CudaOps, rhosvd_sharded, slab_bounds
    x, _, _ = tucker_tensor(spec)
    x32 = philox.round_to_f32(x)
    ranks, p = list(spec.ranks), spec.oversample
    world = 2
    red = ThreadReducer(world)
    results, errors = [None] * world, []

    def run(r):
        c = K.Context(0)
        try:
            start, stop = slab_bounds(spec.dims[-1], world, r)
            xs = tensor_to_dev(np.ascontiguousarray(x32[..., start:stop]), torch.float32)
            results[r] = rhosvd_sharded(CudaOps(c, dev()), xs, spec.dims, start, stop, ranks, p, 0,
                                        allreduce=red.for_rank(r))
            torch.cuda.synchronize()
        except BaseException as e:  # surface in the main thread
            errors.append(e)
            red.barrier.abort()
        finally:
            c.close()

    threads = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    xd = tensor_to_dev(x32, torch.float32)
    core_t, facs_t, res_t = _single_gpu(ctx, xd, spec, K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL)
    ref = _recon(core_t, facs_t, spec.dims, ranks)
    nx = np.linalg.norm(x32)
    for core, facs, rel in results:
        eta = np.linalg.norm(_recon(core, facs, spec.dims, ranks) - ref) / nx
        assert eta <= 1e-5
        # the sharded error value (sums of the slabs' residual passes) against
        # the exact error of the sharded result and the single-GPU value
        e_self, rho = _rho(x32, core, facs, spec.dims, ranks)
        _, rho_t = _rho(x32, core_t, facs_t, spec.dims, ranks)
        check_error_value(rel, res_t["rel_residual"], e_self, eta, rho + rho_t, spec.name)
