"""Bounded device waits (failure detection without a GPU fault).

Every mbarrier wait of the tensor-core kernels has a time limit; a wait that
runs out makes its kernel record KRP_ETIMEOUT in the context's status word,
let its issued copies and MMAs complete, free its tensor memory and return.
Here the limit is set to 1 ns, so the first wait of each kernel that is not
already satisfied runs out (nothing else is changed): the pipeline call must
return KRP_ETIMEOUT, and after the limit is restored the same context must
give the same result as before (the status word cleared, no tensor memory or
copy left behind).  The BF16 form runs every pass over X through those
kernels (the one-pass tree, the core's TTMs, the residual)."""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, tensor_to_dev
from oracle import philox, tucker as TK
from synth import TuckerSpec, tucker_tensor

pytestmark = pytest.mark.gpu


def _run(ctx, xd, spec):
    import torch
    import paper_2507_23207_gb300 as K
    ranks = list(spec.ranks)
    core = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device=dev())
    facs = [torch.empty(n * r, dtype=torch.float64, device=dev()) for n, r in zip(spec.dims, ranks)]
    res = K.krp_tucker_rhosvd(ctx, xd, spec.dims, ranks, spec.oversample, 0,
                              K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL, core, facs)
    torch.cuda.synchronize()
    g = core.cpu().numpy().astype(np.float64).reshape(ranks[::-1]).T
    qs = [f.cpu().numpy().reshape(r, n).T for f, n, r in zip(facs, spec.dims, ranks)]
    return g, qs, res


@pytest.mark.parametrize("form", ["bf16", "bf16x2"])
def test_expired_wait_reports_timeout_and_context_recovers(form):
    torch = require_gpu()
    import paper_2507_23207_gb300 as K
    spec = TuckerSpec("expiry", (256, 96, 40), (4, 4, 4), 1e-3, None, 71, (4, 4, 4), (8, 8, 8))
    x, _, _ = tucker_tensor(spec)
    x32 = philox.round_to_f32(x)
    ctx = K.Context(0)
    try:
        if form == "bf16":
            xd = tensor_to_dev(philox.round_to_bf16(x32), torch.bfloat16)
        else:
            xd = K.krp_split_bf16x2(ctx, tensor_to_dev(x32, torch.float32))
        g0, q0, r0 = _run(ctx, xd, spec)
        ctx.set_wait_limit(1)
        with pytest.raises(K.KrpError) as e:
            _run(ctx, xd, spec)
        assert e.value.status == K.KRP_ETIMEOUT, str(e.value)
        ctx.set_wait_limit(0)
        g1, q1, r1 = _run(ctx, xd, spec)
        # the same result as before the expired call, up to the order of the
        # FP32 atomics of the split reductions (within the reconstruction
        # bound P2 of the parity tests; a damaged context gives garbage)
        nx = np.linalg.norm(x32)
        assert np.linalg.norm(TK.reconstruct(g1, q1) - TK.reconstruct(g0, q0)) <= 1e-5 * nx
        assert abs(r1["rel_residual"] - r0["rel_residual"]) <= 1e-3 * r0["rel_residual"]
        for q in q1:
            assert np.linalg.norm(q.T @ q - np.eye(q.shape[1])) <= 1e-12
    finally:
        ctx.set_wait_limit(0)
        ctx.close()
