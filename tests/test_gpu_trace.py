"""The launch trace (krp_trace_begin / krp_trace_end) over the FP32 form of
RHOSVD-KRP-MEMO, whose FP64 QR runs on a second stream beside the TF32 TTMs:
every launch is listed once with a duration measured on its own stream, and
the traced call gives the same result as an untraced one."""

import json

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, tensor_to_dev
from oracle import philox
from synth import TuckerSpec, tucker_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


def test_trace_of_fp32_step_with_side_stream_qr(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    spec = TuckerSpec("trace", (256, 96, 40), (6, 5, 4), 1e-3, None, 77, (6, 5, 4), (14, 13, 12))
    x, _, _ = tucker_tensor(spec)
    xd = tensor_to_dev(philox.round_to_f32(x), torch.float32)
    ranks = list(spec.ranks)
    flags = K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL

    def run():
        core = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device=dev())
        facs = [torch.empty(n * r, dtype=torch.float64, device=dev()) for n, r in zip(spec.dims, ranks)]
        res = K.krp_tucker_rhosvd(ctx, xd, spec.dims, ranks, spec.oversample, 5, flags, core, facs)
        torch.cuda.synchronize()
        return core.cpu().numpy(), [f.cpu().numpy() for f in facs], res

    g0, q0, r0 = run()
    l0 = ctx.launch_count()
    K.krp_trace_begin(ctx)
    g1, q1, r1 = run()
    tr = K.krp_trace_end(ctx)
    launches = ctx.launch_count() - l0
    names = [n for n, _ in tr]
    # one entry per launch, each with a finite non-negative duration
    assert len(tr) == launches, (len(tr), launches)
    assert all(np.isfinite(t) and t >= 0.0 for _, t in tr)
    json.dumps(tr)
    # the contractions over X on tensor cores, the QR on the second stream
    assert "tc_mttkrp_tf32" in names and "tc_gemm_tn_tf32" in names
    assert "tc_residual_tf32" in names
    assert any("cholqr" in n for n in names)
    # same result traced and untraced (FP32 atomics: rounding order only)
    assert np.linalg.norm(g1 - g0) <= 1e-5 * np.linalg.norm(g0)
    for a, b in zip(q1, q0):
        qa, qb = a.reshape(-1), b.reshape(-1)
        assert np.abs(np.abs(qa) - np.abs(qb)).max() <= 1e-5
    assert abs(r1["rel_residual"] - r0["rel_residual"]) <= 1e-5 * r0["rel_residual"]
