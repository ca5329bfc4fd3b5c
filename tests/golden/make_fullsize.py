"""Write fullsize_c3_c4.json: FP64 oracle results for the two full-size
workloads whose oracle values are affordable on the host.

200^4 decaying-core Tucker tensor (noise-free).  X = G0 x_1 U_1 ... x_4 U_4 with
orthonormal U_i, so by the mixed-product property the mode-i sketch is
Y_i = X_(i) K_i = U_i G0_(i) (kr_{j != i} U_j^T Omega_j): RHOSVD-KRP on X equals
RHOSVD-KRP on the 40^4 core G0 with the factors U_j^T Omega_j, with
Q_i = U_i Q~_i and the same core and reconstruction error.  The script runs
the oracle on that compressed problem with the exact full-size Philox factors
(rounded to FP32 or BF16 as each GPU form uses them), plus the truncated HOSVD
of G0 (= that of X) for reference.

1024 x 1024 block Hankel (128 x 128 blocks of 8 x 8, state order 40).  Alg. 6 on
the explicit matrix with FP32 factors, and on the BF16-rounded blocks with BF16
factors; errors against the matrix each form is given and against the exact one.

Only oracle/ and the seeded input generators are used.  Run from the repo root:
    python tests/golden/make_fullsize.py
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import hankel as HK  # noqa: E402
from oracle import linalg as LA  # noqa: E402
from oracle import philox  # noqa: E402
from oracle import tensor as T  # noqa: E402
from oracle import tucker as TK  # noqa: E402
from synth import config_spec  # noqa: E402
from synth.hankel import hankel_config_spec, markov_parameters  # noqa: E402
from synth.tucker import tucker_factors  # noqa: E402


def compressed_rhosvd_memo(g0, us, dims, seed, ells, ranks, form):
    """RHOSVD-KRP-MEMO of X = G0 x {U_i} (orthonormal U_i), run on G0.

    The mode-i sketch of X is U_i times the mode-i sketch of G0 with the
    factors U_j^T Omega_j (mixed product), so Q_i = U_i Q~_i, the core is the
    same and ||X - X_hat|| = ||G0 - G0_hat||.  Returns the rank-l and the
    truncated relative errors and the truncated core's norm.
    """
    d = len(dims)
    oms = TK.memo_factors(seed, dims, max(ells), omega_round=form)
    omt = [u.T @ om for u, om in zip(us, oms)]
    qs = []
    for i in range(d):
        om_i = [omt[j][:, :ells[i]] if j != i else None for j in range(d)]
        q, _ = LA.householder_qr(T.mttkrp(g0, om_i, i))
        qs.append(q)
    g = T.multi_ttm(g0, [q.T for q in qs])
    g2, q2 = TK.truncate_core(g, qs, ranks)
    return TK.rel_error(g0, g, qs), TK.rel_error(g0, g2, q2), float(T.frob(g2))


def c3_values():
    spec = config_spec("c3")
    g0, us = tucker_factors(spec)
    ells, ranks = list(spec.ell), list(spec.ranks)
    out = {"workload": "200^4 Tucker, core 40^4 N(0,1)*0.8^(i+j+k+l), no noise, "
                       "RHOSVD-KRP-MEMO l=30, truncated to rank 20",
           "dims": list(spec.dims), "ell": ells, "ranks": ranks,
           "x_norm": float(T.frob(g0))}
    gh, qh = TK.hosvd(g0, ranks)
    out["hosvd_rel_error"] = TK.rel_error(g0, gh, qh)
    for form in ("f32", "bf16"):
        e_l, e_r, gn = compressed_rhosvd_memo(g0, us, spec.dims, spec.omega_seed, ells, ranks,
                                              form)
        out[f"rhosvd_memo_rank_l_rel_error_{form}"] = e_l
        out[f"rhosvd_memo_truncated_rel_error_{form}"] = e_r
        out[f"core_norm_truncated_{form}"] = gn
    return out


def c4_values():
    spec = hankel_config_spec("c4")
    blocks = markov_parameters(spec)
    h = HK.block_hankel(blocks)
    hn = float(np.linalg.norm(h))
    out = {"workload": "1024x1024 block Hankel, 128x128 blocks of 8x8, state order 40, "
                       "Alg. 6 with l_r=50, l_l=75, r=40",
           "h_norm": hn}
    for form in ("f32", "bf16"):
        b = philox.round_to_f32(blocks) if form == "f32" else philox.round_to_bf16(blocks)
        hb = HK.block_hankel(b)
        res = HK.single_pass_svd(b, spec.r, spec.ell_r, spec.ell_l, spec.omega_seed,
                                 omega_round=form)
        approx = res["U"] @ np.diag(res["S"]) @ res["V"].T
        out[f"rel_error_vs_input_{form}"] = float(np.linalg.norm(hb - approx) / np.linalg.norm(hb))
        out[f"rel_error_vs_exact_{form}"] = float(np.linalg.norm(h - approx) / hn)
        out[f"sigma_{form}"] = [float(v) for v in res["S"]]
    return out


def main():
    t0 = time.time()
    vals = {"c3": c3_values()}
    t1 = time.time()
    vals["c4"] = c4_values()
    t2 = time.time()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_c3_c4.json")
    with open(path, "w") as f:
        json.dump(vals, f, indent=1)
    print(f"wrote {path} (c3 {t1 - t0:.1f} s, c4 {t2 - t1:.1f} s)")


if __name__ == "__main__":
    main()
