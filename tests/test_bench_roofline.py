"""bench.py's roofline object on a synthetic launch trace (CPU): the dominant
kernel is the one with the largest share of the timed steps among those
that read all of X, `achieved` is its algorithmic bytes over its average
launch time, and the other candidates are reported beside it."""

import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as B
    return B


def _spec():
    return SimpleNamespace(numel=1024 ** 3, ell=(48, 48, 48), ranks=(32, 32, 32),
                           dims=(1024, 1024, 1024))


def test_dominant_kernel_and_beside(bench, monkeypatch):
    monkeypatch.setattr(bench, "sm_count", lambda: 152)
    steps = 2
    per_step = [("gen_factors", 0.02), ("tc_mttkrp_tf32", 0.95), ("tc_gemm_tn_tf32", 0.92),
                ("diag_mid_f32", 0.05), ("cholqr_jobs_gram_f64", 0.01),
                ("tc_gemm_tn_tf32", 0.92), ("gemm_tn_tile<48>", 0.08),
                ("tc_residual_tf32", 0.70)]
    f32 = {"trace": per_step * steps, "ms": 4.75, "clocks": {"sm_max_mhz": 2070.0}}
    peaks = {"hbm_gbs": 6794.5}
    out = bench.trace_roofline(_spec(), f32, peaks, SimpleNamespace(steps=steps))
    # the TTM: two launches per step, 1.84 ms of the step
    assert out["kernel"].startswith("tc_gemm_tn_tf32_kernel")
    assert out["bound"] == "hbm" and out["unit"] == "GB/s" and out["peak"] == 6794.5
    n, ell = 1024 ** 3, 48
    work = n * 4.0 + n / 1024 * ell * 4.0
    assert out["achieved"] == pytest.approx(work / 0.92e-3 / 1e9, rel=1e-3)
    assert out["frac"] == pytest.approx(out["achieved"] / 6794.5, rel=1e-3)
    assert out["launches_averaged"] == 2 * steps
    assert out["kernel_share_of_step"] == pytest.approx(1.84 / 4.75, rel=1e-3)
    assert out["traffic"] == pytest.approx(bench.TRAFFIC_1024["tc_gemm_tn_tf32"])
    assert set(out["beside"]) == {"tc_mttkrp_tf32", "tc_residual_tf32"}
    m = out["beside"]["tc_mttkrp_tf32"]
    assert m["achieved"] == pytest.approx((n * 4.0 + 1024 * ell * 4.0) / 0.95e-3 / 1e9, rel=1e-3)


def test_big_launches_drop_the_small_ones(bench):
    # two X-sized launches per step and one small launch of the same kernel
    times = [0.9, 0.1, 0.92, 0.91, 0.12, 0.9]
    big = bench._big_launches(times, steps=2)
    assert sorted(big) == [0.9, 0.9, 0.91, 0.92]


def test_no_candidate_in_the_trace(bench, monkeypatch):
    monkeypatch.setattr(bench, "sm_count", lambda: 152)
    f32 = {"trace": [("gen_factors", 0.02)], "ms": 1.0}
    out = bench.trace_roofline(_spec(), f32, {"hbm_gbs": 6794.5}, SimpleNamespace(steps=1))
    assert "error" in out
