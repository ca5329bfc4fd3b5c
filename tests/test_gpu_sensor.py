"""Sensor placement (Sec. 6) on the GPU against the oracle.

* Selection: on the same orthonormal factors Q_i (Haar draws, 150 x 12,
  90 x 10, 60 x 8), the sensor indices are bit-exact with the oracle's
  pivoted QR (inputs whose pivot decisions have a relative margin > 1e-9, so
  the FP64 decisions cannot flip under another summation order), and the
  interpolation factors A_i agree to 1e-12 relative; A_i is the identity on
  the sensors.
* Reconstruction: T_hat x {A_i} against the oracle's on the same T_hat and
  the same (oracle) factors, to FP32 output rounding (1e-6 relative).
* The paper's training/test pipeline on synthetic snapshots (the flow data
  set is not available): RHOSVD-KRP-MEMO of the training snapshots on the
  GPU, selection from its spatial factors, reconstruction of held-out
  snapshots from their values on the sensor grid; the test-phase error is
  within 2x (+1e-6) of the same pipeline run by the oracle on the host.
"""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, tensor_to_dev, mat_to_dev, mat_from_dev
from oracle import philox, sensor as SE, tucker as TK
from synth import TuckerSpec, haar, tucker_tensor

pytestmark = pytest.mark.gpu

DIMS, ELLS = (150, 90, 60), (12, 10, 8)


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


def _factors(seed):
    rng = np.random.default_rng(seed)
    qs = [haar(n, l, rng) for n, l in zip(DIMS, ELLS)]
    for q in qs:
        assert SE.pivot_margins(q).min() > 1e-9
    return qs


def _select(ctx, qs):
    import torch
    import paper_2507_23207_gb300 as K
    qd = [mat_to_dev(q, torch.float64) for q in qs]
    idx = [torch.empty(l, dtype=torch.int32, device=dev()) for l in ELLS]
    A = [torch.empty((l, n), dtype=torch.float64, device=dev()) for n, l in zip(DIMS, ELLS)]
    K.krp_sensor_select(ctx, DIMS, ELLS, qd, idx, A)
    torch.cuda.synchronize()
    return [i.cpu().numpy() for i in idx], [mat_from_dev(a, n, l) for a, n, l in zip(A, DIMS, ELLS)]


@pytest.mark.parametrize("seed", [61, 62])
def test_select_matches_oracle(ctx, seed):
    qs = _factors(seed)
    idx_g, a_g = _select(ctx, qs)
    for q, ig, ag in zip(qs, idx_g, a_g):
        io = SE.pivoted_qr_select(q)
        assert np.array_equal(ig, io)
        ao = SE.interpolation_factor(q, io)
        assert np.linalg.norm(ag - ao) <= 1e-12 * np.linalg.norm(ao)
        assert np.linalg.norm(ag[ig, :] - np.eye(q.shape[1])) <= 1e-12


def test_reconstruct_matches_oracle(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    qs = _factors(63)
    idx = [SE.pivoted_qr_select(q) for q in qs]
    a = [SE.interpolation_factor(q, i) for q, i in zip(qs, idx)]
    t_hat = philox.round_to_f32(np.random.default_rng(5).standard_normal(ELLS))
    out = torch.empty(int(np.prod(DIMS)), dtype=torch.float32, device=dev())
    K.krp_sensor_reconstruct(ctx, DIMS, ELLS, [mat_to_dev(x, torch.float64) for x in a],
                             tensor_to_dev(t_hat, torch.float32), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64).reshape(DIMS[::-1]).T
    ref = SE.sensor_reconstruct(t_hat, a)
    assert np.linalg.norm(got - ref) <= 1e-6 * np.linalg.norm(ref)


def test_training_and_test_pipeline(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    dims, n_train = (60, 45, 30, 50), 40
    spec = TuckerSpec("snapshots", dims, (6, 5, 4, 8), 1e-4, None, 71, (6, 5, 4, 8), (10, 9, 8, 12))
    s, _, _ = tucker_tensor(spec)
    s = philox.round_to_f32(s)
    train = np.asfortranarray(s[..., :n_train])
    test = s[..., n_train:]
    tdims = dims[:3] + (n_train,)
    ells = [r + 4 for r in spec.ranks]
    core = torch.empty(int(np.prod(ells)), dtype=torch.float32, device=dev())
    facs = [torch.empty(n * c, dtype=torch.float64, device=dev()) for n, c in zip(tdims, ells)]
    K.krp_tucker_rhosvd(ctx, tensor_to_dev(train, torch.float32), tdims, spec.ranks, 4, 0,
                        K.KRP_MEMO, core, facs)
    sp_ells = ells[:3]
    idx = [torch.empty(l, dtype=torch.int32, device=dev()) for l in sp_ells]
    A = [torch.empty((l, n), dtype=torch.float64, device=dev()) for n, l in zip(dims[:3], sp_ells)]
    K.krp_sensor_select(ctx, dims[:3], sp_ells, facs[:3], idx, A)
    torch.cuda.synchronize()
    ig = [i.cpu().numpy() for i in idx]
    err_g = []
    out = torch.empty(int(np.prod(dims[:3])), dtype=torch.float32, device=dev())
    for t in range(test.shape[3]):
        field = test[..., t]
        t_hat = np.asfortranarray(field[np.ix_(*ig)])
        K.krp_sensor_reconstruct(ctx, dims[:3], sp_ells, A, tensor_to_dev(t_hat, torch.float32), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64).reshape(dims[:3][::-1]).T
        err_g.append(np.linalg.norm(got - field) / np.linalg.norm(field))
        assert np.allclose(got[np.ix_(*ig)], t_hat, rtol=0, atol=1e-5 * np.abs(t_hat).max())
    # the oracle: the same pipeline on the host
    ora = TK.rhosvd_krp(train, ells, 0, memo=True, omega_round="f32")
    io = [SE.pivoted_qr_select(q) for q in ora["Q"][:3]]
    ao = [SE.interpolation_factor(q, i) for q, i in zip(ora["Q"][:3], io)]
    err_o = []
    for t in range(test.shape[3]):
        field = test[..., t]
        rec = SE.sensor_reconstruct(field[np.ix_(*io)], ao)
        err_o.append(np.linalg.norm(rec - field) / np.linalg.norm(field))
    assert max(err_g) <= 2.0 * max(err_o) + 1e-6, (max(err_g), max(err_o))
    assert np.mean(err_g) <= 2.0 * np.mean(err_o) + 1e-6


def test_select_rejects_bad_arguments(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    q = mat_to_dev(haar(10, 3, np.random.default_rng(1)), torch.float64)
    idx = torch.empty(4, dtype=torch.int32, device=dev())
    A = torch.empty((4, 10), dtype=torch.float64, device=dev())
    for dims, ells in (((10,), (11,)), ((10,), (65,)), ((10,), (0,))):
        with pytest.raises(K.KrpError) as e:
            K.krp_sensor_select(ctx, dims, ells, [q], [idx], [A])
        assert e.value.status == K.KRP_EINVAL
