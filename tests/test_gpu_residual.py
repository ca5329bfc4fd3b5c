"""The residual pass (||X - G x_1 Q_1 ... x_d Q_d||_F^2 and ||X||_F^2, the
relative error of Sec. 3's approximations) through the krp_residual entry
point, on the shapes where it changes kernels: the FP32 form's mode-1 stage
runs on the tensor cores for n_1 % 4 == 0 and c_1 <= 32 (c_1 = 32 is the
widest), and on the CUDA cores otherwise (c_1 = 33, n_1 odd).  Row and column
counts are ragged against the 128 x 128 tiles.  The expected values are
FP64 sums over the same FP32 X, core and factors; the tolerance is the
rounding model of tests/parity.py."""

import math

import numpy as np
import pytest

from tests.gpu_util import require_gpu, dev, tensor_to_dev
from tests.parity import U_F32, U_TF32_PAIR, eval_bound
from oracle import philox, tucker as TK

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    require_gpu()
    import paper_2507_23207_gb300 as K
    c = K.Context(0)
    yield c
    c.close()


CASES = [
    ((260, 36, 20), (32, 6, 5), 1e-3),   # tensor-core mode-1 stage, widest c_1, ragged tiles
    ((132, 21, 13), (4, 3, 3), 1e-5),    # tensor-core, small error
    ((128, 128, 9), (12, 10, 4), 1e-3),  # tensor-core, whole tiles
    ((260, 36, 20), (33, 6, 5), 1e-3),   # c_1 > 32: CUDA-core mode-1 stage
    ((257, 30, 11), (8, 5, 4), 1e-3),    # n_1 % 4 != 0: CUDA-core mode-1 stage
]


def _problem(dims, cdims, noise, seed):
    rng = np.random.default_rng(seed)
    qs = [np.linalg.qr(rng.standard_normal((n, c)))[0] for n, c in zip(dims, cdims)]
    g = philox.round_to_f32(rng.standard_normal(cdims) * np.geomspace(1.0, 0.1, cdims[0])[
        (slice(None),) + (None,) * (len(dims) - 1)])
    x = TK.reconstruct(g, qs)
    x = x + noise * np.linalg.norm(x) / math.sqrt(x.size) * rng.standard_normal(dims)
    return philox.round_to_f32(x), g, qs


@pytest.mark.parametrize("dims,cdims,noise", CASES)
def test_residual_matches_fp64_sums(ctx, dims, cdims, noise):
    import torch
    import paper_2507_23207_gb300 as K
    require_gpu()
    x, g, qs = _problem(dims, cdims, noise, 97 + sum(dims) + sum(cdims))
    xd = tensor_to_dev(x, torch.float32)
    core = torch.from_numpy(np.ascontiguousarray(g.T).reshape(-1).astype(np.float32)).to(dev())
    facs = [torch.from_numpy(np.ascontiguousarray(q.T).reshape(-1)).to(dev()) for q in qs]
    d2, x2 = K.krp_residual(ctx, xd, dims, cdims, core, facs)
    torch.cuda.synchronize()
    x64 = x.astype(np.float64)
    nx2 = float(np.sum(x64 * x64))
    assert abs(x2 - nx2) <= 128 * 2.0 ** -24 * nx2
    xh = TK.reconstruct(g, qs)
    e_self = math.sqrt(float(np.sum((x64 - xh) ** 2)) / nx2)
    e_gpu = math.sqrt(d2 / x2)
    tensor_core = dims[0] % 4 == 0 and cdims[0] <= 32
    rho = eval_bound(cdims, dims, np.linalg.norm(xh) / math.sqrt(nx2), e_self, U_F32,
                     U_TF32_PAIR if tensor_core else U_F32)
    assert abs(e_gpu - e_self) <= 1e-5 * e_self + rho, (dims, cdims, e_gpu, e_self, rho)
    print(f"{dims} c={cdims}: e_self {e_self:.6e} |e_gpu - e_self| {abs(e_gpu - e_self):.2e} "
          f"rho {rho:.2e}")
