"""a6-a8 parity: RHOSVD-KRP (fresh, memoized), RSTHOSVD-KRP, truncation, residual.

Compared quantities (basis-invariant, FP32 bound 1e-5):
  P2  ||X_hat_gpu - X_hat_oracle||_F / ||X||_F
  P3  |e_gpu - e_oracle| with e = ||X - X_hat||_F / ||X||_F: 1e-5 relative,
      widened by the measured P2 distance and the residual pass's rounding
      bound where FP32 cannot resolve e to 1e-5 (tests/parity.py)
  P4  after truncation, the rank-r projectors Q_r Q_r^T of every mode
plus orthonormality of every returned factor (FP64 QR).  The oracle runs the
same algorithm on the same FP32-rounded X with its own FP32-rounded factors.
"""

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, tensor_to_dev, rel
from tests.parity import U_F32, U_TF32_PAIR, check_error_value, eval_bound
from oracle import philox, tucker as TK
from synth import TuckerSpec, tucker_tensor, config_spec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


def run_gpu(ctx, x32, spec_dims, ranks, p, seed, flags, sequential=False, host=False):
    import torch
    import paper_2507_23207_gb300 as K
    trunc = bool(flags & K.KRP_TRUNCATE)
    oc = [r if trunc else r + p for r in ranks]
    if host:
        from synth import to_torch_layout
        xd = to_torch_layout(np.asfortranarray(x32)).to(torch.float32)
        core = torch.empty(int(np.prod(oc)), dtype=torch.float32)
        facs = [torch.empty(n * c, dtype=torch.float64) for n, c in zip(spec_dims, oc)]
    else:
        xd = tensor_to_dev(x32, torch.float32)
        core = torch.empty(int(np.prod(oc)), dtype=torch.float32, device=dev())
        facs = [torch.empty(n * c, dtype=torch.float64, device=dev()) for n, c in zip(spec_dims, oc)]
    fn = K.krp_tucker_sthosvd if sequential else K.krp_tucker_rhosvd
    res = fn(ctx, xd, spec_dims, ranks, p, seed, flags, core, facs)
    torch.cuda.synchronize()
    g = core.cpu().numpy().reshape(oc[::-1]).T.astype(np.float64)
    qs = [f.cpu().numpy().reshape(c, n).T for f, n, c in zip(facs, spec_dims, oc)]
    return g, qs, res


def oracle_run(x32, ells, seed, memo, sequential):
    if sequential:
        # step 0 sketches the FP32 X with FP32 factors; later steps sketch FP32 cores
        return TK.rsthosvd_krp(x32, ells, seed, omega_round="f32")
    return TK.rhosvd_krp(x32, ells, seed, memo=memo, omega_round="f32")


SPECS = [
    TuckerSpec("c1", (64, 64, 64), (5, 5, 5), 1e-6, None, 1001, (5, 5, 5), (10, 10, 10)),
    TuckerSpec("ragged", (37, 29, 23), (3, 4, 5), 1e-3, None, 17, (3, 4, 5), (6, 7, 8)),
    TuckerSpec("d4", (12, 10, 9, 8), (3, 3, 2, 3), 1e-2, None, 23, (3, 3, 2, 3), (5, 5, 4, 5)),
    TuckerSpec("tall", (300, 20, 10), (6, 5, 4), 1e-4, None, 29, (6, 5, 4), (10, 9, 8)),
    # n_1 % 4 == 0 with a 4-row ragged 128-row block, c % 4 == 0 and
    # S = 21 * 13 not a multiple of 64: the persistent tiled residual path
    TuckerSpec("tiled", (132, 21, 13), (4, 3, 3), 1e-3, None, 31, (4, 3, 3), (8, 7, 7)),
    # a matrix (d = 2) and a sketch as wide as its mode (l_i = n_i).  The
    # truncated projectors are compared to 1e-5, and their sensitivity to
    # FP32 rounding grows as 1 / (sigma_r - sigma_r+1): the matrix's data seed
    # gives sigma_3 / sigma_1 = 0.63 (seed 37 gave 0.009, where the oracle
    # itself moves the projectors by ~4e-5 under FP32-level perturbations)
    TuckerSpec("matrix", (50, 40), (3, 3), 1e-3, None, 40, (3, 3), (6, 6)),
    TuckerSpec("l_eq_n", (8, 8, 8), (4, 4, 4), 1e-3, None, 39, (4, 4, 4), (8, 8, 8)),
]


@pytest.mark.parametrize("spec", SPECS, ids=[s.name for s in SPECS])
@pytest.mark.parametrize("variant", ["fresh", "memo", "sthosvd"])
def test_tucker_parity(ctx, spec, variant):
    import paper_2507_23207_gb300 as K
    x, _, _ = tucker_tensor(spec)
    x32 = philox.round_to_f32(x)
    p = spec.oversample
    ells = [r + p for r in spec.ranks]
    memo = variant == "memo"
    seq = variant == "sthosvd"
    flags = (K.KRP_MEMO if memo else 0) | K.KRP_RESIDUAL
    g, qs, res = run_gpu(ctx, x32, spec.dims, spec.ranks, p, spec.omega_seed, flags, seq)
    ora = oracle_run(x32, ells, spec.omega_seed, memo, seq)
    for q in qs:
        assert np.linalg.norm(q.T @ q - np.eye(q.shape[1])) <= 1e-12
    nx = np.linalg.norm(x32)
    _check_p2_p3(x32, g, qs, ora["G"], ora["Q"], res["rel_residual"], spec.dims,
                 f"{spec.name}/{variant}")
    assert abs(res["x_norm"] - nx) <= 1e-6 * nx
    # truncated variant
    flags_t = flags | K.KRP_TRUNCATE
    g2, q2, res2 = run_gpu(ctx, x32, spec.dims, spec.ranks, p, spec.omega_seed, flags_t, seq)
    g2o, q2o = TK.truncate_core(ora["G"], ora["Q"], spec.ranks)
    for a, b in zip(q2, q2o):
        assert np.linalg.norm(a @ a.T - b @ b.T) / np.sqrt(a.shape[1]) <= 1e-5
    _check_p2_p3(x32, g2, q2, g2o, q2o, res2["rel_residual"], spec.dims,
                 f"{spec.name}/{variant}/truncated")
    assert list(res2["core_dims"]) == list(spec.ranks)


def _check_p2_p3(x, g, qs, g_o, q_o, e_gpu, dims, what, p2_tol=1e-5, unit=U_F32,
                 unit1=U_TF32_PAIR):
    """P2 (reconstructions within p2_tol of ||X||) and P3 (error values, with
    the bound of tests/parity.py); returns the measured P2 distance."""
    nx = np.linalg.norm(x)
    xh = TK.reconstruct(g, qs)
    eta = np.linalg.norm(xh - TK.reconstruct(g_o, q_o)) / nx
    assert eta <= p2_tol, (what, eta)
    e_self = TK.rel_error(x, g, qs)
    e_ora = TK.rel_error(x, g_o, q_o)
    rho = eval_bound(g.shape, dims, np.linalg.norm(xh) / nx, e_self, unit, unit1)
    check_error_value(e_gpu, e_ora, e_self, eta, rho, what)
    return eta


def test_exact_recovery_fp32(ctx):
    import paper_2507_23207_gb300 as K
    spec = TuckerSpec("exact", (40, 36, 30), (4, 3, 5), 0.0, None, 31, (4, 3, 5), (7, 6, 8))
    x, _, _ = tucker_tensor(spec)
    x32 = philox.round_to_f32(x)
    for flags in (K.KRP_MEMO | K.KRP_RESIDUAL, K.KRP_RESIDUAL | K.KRP_TRUNCATE):
        g, qs, res = run_gpu(ctx, x32, spec.dims, spec.ranks, spec.oversample, 0, flags)
        # FP32 arithmetic floor: the error of an exact-rank input is ~FP32 epsilon
        assert res["rel_residual"] <= 1e-5


def test_host_pointers_match_device_pointers(ctx):
    import paper_2507_23207_gb300 as K
    spec = SPECS[1]
    x, _, _ = tucker_tensor(spec)
    x32 = philox.round_to_f32(x)
    flags = K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL
    gd, qd, rd = run_gpu(ctx, x32, spec.dims, spec.ranks, spec.oversample, 0, flags)
    gh, qh, rh = run_gpu(ctx, x32, spec.dims, spec.ranks, spec.oversample, 0, flags, host=True)
    # split-K reductions use atomics, so two runs agree to FP32 rounding, not bitwise
    nx = np.linalg.norm(x32)
    xd, xh = TK.reconstruct(gd, qd), TK.reconstruct(gh, qh)
    eta = np.linalg.norm(xd - xh) / nx
    assert eta <= 1e-6
    # both error values are within the residual pass's rounding bound of the
    # exact errors of their own results, which differ by at most eta
    e_self = TK.rel_error(x32, gd, qd)
    rho = eval_bound(gd.shape, spec.dims, np.linalg.norm(xd) / nx, e_self, U_F32, U_TF32_PAIR)
    assert abs(rd["rel_residual"] - rh["rel_residual"]) <= 2e-5 * e_self + eta + 2 * rho


def test_timings_reported(ctx):
    import paper_2507_23207_gb300 as K
    spec = SPECS[0]
    x, _, _ = tucker_tensor(spec)
    x32 = philox.round_to_f32(x)
    for seq in (False, True):
        _, _, res = run_gpu(ctx, x32, spec.dims, spec.ranks, spec.oversample, 0,
                            K.KRP_MEMO | K.KRP_TIMINGS | K.KRP_TRUNCATE | K.KRP_RESIDUAL, seq)
        t = res["times"]
        assert t["total_ms"] > 0 and t["sketch_ms"] > 0 and t["qr_ms"] > 0 and t["core_ms"] > 0
        assert t["total_ms"] >= t["sketch_ms"]


def test_tucker_invalid_arguments(ctx):
    import torch
    import paper_2507_23207_gb300 as K
    x32 = np.zeros((8, 8, 8), dtype=np.float64, order="F")
    with pytest.raises(K.KrpError) as e:  # l = 9 > n = 8
        run_gpu(ctx, x32, (8, 8, 8), (5, 5, 5), 4, 0, 0)
    assert e.value.status == K.KRP_EINVAL
    with pytest.raises(K.KrpError):
        run_gpu(ctx, x32, (8, 8, 8), (0, 2, 2), 1, 0, 0)
    with pytest.raises(K.KrpError):
        run_gpu(ctx, x32, (8, 8, 8), (2, 2, 2), 1, 0, 0x100)


@pytest.mark.parametrize("memo", [False, True])
def test_zero_tensor(ctx, memo):
    """X = 0: every sketch is zero, so every QR pivot collapses and the
    columns are refilled; the factors must still be orthonormal, the core and
    the reconstruction zero, and the relative residual defined (0)."""
    import torch
    import paper_2507_23207_gb300 as K
    dims, ranks, p = (16, 12, 10), (2, 2, 2), 2
    ells = [r + p for r in ranks]
    xd = torch.zeros(int(np.prod(dims)), dtype=torch.float32, device=dev())
    for trunc in (False, True):
        out = list(ranks) if trunc else ells
        core = torch.empty(int(np.prod(out)), dtype=torch.float32, device=dev())
        facs = [torch.empty(n * o, dtype=torch.float64, device=dev()) for n, o in zip(dims, out)]
        flags = (K.KRP_MEMO if memo else 0) | K.KRP_RESIDUAL | (K.KRP_TRUNCATE if trunc else 0)
        res = K.krp_tucker_rhosvd(ctx, xd, dims, list(ranks), p, 0, flags, core, facs)
        torch.cuda.synchronize()
        for f, n, o in zip(facs, dims, out):
            q = f.cpu().numpy().reshape(o, n).T
            assert np.all(np.isfinite(q))
            assert np.linalg.norm(q.T @ q - np.eye(o)) <= 1e-12
        assert float(core.abs().max()) == 0.0
        assert res["rel_residual"] == 0.0 and res["x_norm"] == 0.0


def test_host_bf16_input_matches_device_input(ctx):
    """A BF16 tensor in host memory: the library copies it in chunks of the
    last mode on a second stream while it sketches the chunks already on the
    device; the result is the one of the same call on a device copy."""
    import torch
    import paper_2507_23207_gb300 as K
    spec = TuckerSpec("hostbf", (40, 33, 27), (4, 3, 5), 1e-3, None, 63, (4, 3, 5), (8, 7, 9))
    x, _, _ = tucker_tensor(spec)
    xb = philox.round_to_bf16(x)
    from synth import to_torch_layout
    xh = to_torch_layout(np.asfortranarray(xb)).to(torch.bfloat16)
    flags = K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL
    outs = []
    for xx in (xh.pin_memory(), xh.to(dev())):
        ranks = list(spec.ranks)
        core = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device=dev())
        facs = [torch.empty(n * r, dtype=torch.float64, device=dev()) for n, r in zip(spec.dims, ranks)]
        res = K.krp_tucker_rhosvd(ctx, xx, spec.dims, ranks, spec.oversample, 0, flags, core, facs)
        torch.cuda.synchronize()
        g = core.cpu().numpy().reshape(ranks[::-1]).T.astype(np.float64)
        qs = [f.cpu().numpy().reshape(r, n).T for f, n, r in zip(facs, spec.dims, ranks)]
        outs.append((TK.reconstruct(g, qs), res["rel_residual"]))
    nx = np.linalg.norm(xb)
    assert np.linalg.norm(outs[0][0] - outs[1][0]) <= 1e-5 * nx
    assert abs(outs[0][1] - outs[1][1]) <= 1e-3 * outs[1][1]
