"""Benchmark of the KRP randomized-Tucker hot path on one GB300 (or N replicas).

A step is one pass of the whole path over one synthetic tensor, resident in HBM:
factor generation (Philox), the all-mode KRP sketch by dimension tree (MEMO),
FP64 QR of every sketch, the multi-TTM core, FP64 rank-r truncation and the
FP64-accumulated residual ||X - X_hat|| / ||X|| -- i.e. krp_tucker_rhosvd with
KRP_MEMO | KRP_TRUNCATE | KRP_RESIDUAL.

Default workload: the 1024^3 FP32 tensor of multilinear rank 32 + 1e-4 noise,
l = 48 (r = 32, oversampling 16), seed 0.  The BF16 tensor-core form is timed on
the BF16 copy of the same tensor and reported beside it.

Metric: algorithmic GB/s of the step (three passes over X: sketch, core,
residual, N * bytes each), with TFLOP/s from the paper's leading-order flop
counts and the step time.  Prints ONE JSON line.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "KRP sketch GB/s & TFLOP/s, RHOSVD time: BF16 vs FP32 at stated rel. error"


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def sm_count() -> int:
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp32_ffma_peak_tflops(sm_mhz: float, sms: int) -> float:
    # 128 FP32 lanes per SM, one FMA (2 flops) per lane per clock
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- workload --
def make_inputs(spec, device, want_bf16=True):
    import torch
    from synth.tucker import tucker_tensor_device
    x64, _, _ = tucker_tensor_device(spec, device=device)
    x32 = x64.to(torch.float32)
    xbf = x64.to(torch.bfloat16) if want_bf16 else None
    del x64
    torch.cuda.empty_cache()
    return x32, xbf


def step_flops(spec):
    n = spec.numel
    ell = max(spec.ell)
    d = spec.d
    # Table 1 (MEMO): 4 N l for the dimension-tree sketch + the multi-TTM core
    core = 0.0
    size = float(n)
    for i in range(d):
        core += 2.0 * size * spec.ell[i]
        size = size / spec.dims[i] * spec.ell[i]
    sketch = 4.0 * n * ell
    resid = 2.0 * n * spec.ranks[0]
    qr = sum(4.0 * nn * l * l for nn, l in zip(spec.dims, spec.ell))
    return sketch, core, resid, qr


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2507_23207_gb300 as K
    from synth import config_spec

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    spec = workload(args)
    peaks, peak_src = measured_peaks()
    x32, xbf = make_inputs(spec, dev, want_bf16=not args.no_bf16)
    forms = [("f32", x32)] + ([("bf16", xbf)] if xbf is not None else [])
    if xbf is not None:
        ctx0 = K.Context(local_rank, torch.cuda.current_stream(dev).cuda_stream)
        forms.append(("bf16x2", K.krp_split_bf16x2(ctx0, x32)))
        torch.cuda.synchronize()
        ctx0.close()
    ranks = list(spec.ranks)
    p = spec.oversample
    flags = K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL
    core = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device=dev)
    facs = [torch.empty(n * r, dtype=torch.float64, device=dev) for n, r in zip(spec.dims, ranks)]
    stream = torch.cuda.current_stream(dev)
    ctx = K.Context(local_rank, stream.cuda_stream)
    sk, co, rs, qr = step_flops(spec)
    results = {}
    for form, x in forms:
        def step(fl=flags):
            return K.krp_tucker_rhosvd(ctx, x, spec.dims, ranks, p, spec.omega_seed, fl, core, facs)
        for _ in range(args.warmup):
            res = step()
        # phase breakdown (separate, synchronising run)
        ph = step(flags | K.KRP_TIMINGS)["times"]
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        launches0 = ctx.launch_count()
        clocks = ClockSampler(local_rank)
        clocks.start()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        if form == "f32":
            K.krp_trace_begin(ctx)  # an event after every launch, for the roofline
        ev0.record(stream)
        for _ in range(args.steps):
            res = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        trace = K.krp_trace_end(ctx) if form == "f32" else None
        clk = clocks.stop()
        ms = ev0.elapsed_time(ev1) / args.steps
        launches = (ctx.launch_count() - launches0)
        if world > 1:
            t = torch.tensor([ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        results[form] = {"ms": ms, "res": res, "phases": ph, "clocks": clk, "trace": trace,
                         "launches": launches,
                         "bytes_per_elem": 4 if form == "bf16x2" else x.element_size()}
    # dominant-kernel roofline from the launch trace of the timed FP32 steps
    kr = trace_roofline(spec, results["f32"], peaks, args)
    sketch = sketch_rooflines(ctx, spec, forms, dev, stream, peaks, results["f32"]["clocks"], args)
    # e2e through the C ABI with host buffers (pinned), FP32 form
    e2e = e2e_run(ctx, spec, x32, args) if rank == 0 and not args.no_e2e else None
    extra = {}
    if not args.no_extra and not args.dims and args.config == "c2":
        extra["sthosvd_1024cubed"] = sthosvd_run(ctx, spec, forms, dev, stream, args)
        del forms, x, x32, xbf
        torch.cuda.empty_cache()
        extra["tucker_200pow4"] = c3_run(ctx, dev, stream, args)
        extra["block_hankel_1024"] = c4_run(ctx, dev, stream, args)
        extra["batched_512_tucker"] = batch_run(ctx, dev, stream, args)
        extra["batched_64_hankel"] = hankel_batch_run(ctx, dev, stream, args)
    ctx.close()
    return spec, results, kr, sketch, e2e, peaks, peak_src, (sk, co, rs, qr), extra


def _timed(stream, step, reps, warm):
    import torch
    for _ in range(warm):
        res = step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        res = step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, res


def _golden():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                        "fullsize_c3_c4.json")
    with open(path) as f:
        return json.load(f)


def sthosvd_run(ctx, spec, forms, dev, stream, args):
    """RSTHOSVD-KRP (Alg. 8) + truncation + residual on the same 1024^3 tensors."""
    import torch
    import paper_2507_23207_gb300 as K
    ranks = list(spec.ranks)
    core = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device=dev)
    facs = [torch.empty(n * r, dtype=torch.float64, device=dev) for n, r in zip(spec.dims, ranks)]
    flags = K.KRP_TRUNCATE | K.KRP_RESIDUAL
    out = {}
    for form, x in forms:
        ms, res = _timed(stream, lambda: K.krp_tucker_sthosvd(
            ctx, x, spec.dims, ranks, spec.oversample, spec.omega_seed, flags, core, facs),
            reps=max(3, min(args.steps, 5)), warm=2)
        out[form] = {"ms": round(ms, 3), "rel_error": res["rel_residual"],
                     "gbs": round(3.0 * spec.numel * x.element_size() / (ms * 1e-3) / 1e9, 1)}
    out["note"] = "steps: sketch+TTM of mode 1 on X, then the shrinking core; residual pass on X"
    return out


def c3_run(ctx, dev, stream, args):
    """200^4 decaying-core workload, RHOSVD-KRP-MEMO l=30 -> rank 20, both forms,
    next to the FP64 oracle's errors (stored by tests/golden/make_fullsize.py)."""
    import torch
    import paper_2507_23207_gb300 as K
    from synth import config_spec
    from synth.tucker import tucker_tensor_device
    spec = config_spec("c3")
    x64, _, _ = tucker_tensor_device(spec, device=dev)
    xs = {"f32": x64.to(torch.float32), "bf16": x64.to(torch.bfloat16)}
    del x64
    torch.cuda.empty_cache()
    xs["bf16x2"] = K.krp_split_bf16x2(ctx, xs["f32"])
    ranks = list(spec.ranks)
    core = torch.empty(int(np.prod(ranks)), dtype=torch.float32, device=dev)
    facs = [torch.empty(n * r, dtype=torch.float64, device=dev) for n, r in zip(spec.dims, ranks)]
    flags = K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL
    gold = _golden()["c3"]
    out = {"workload": "200x200x200x200, core 40^4 N(0,1)*0.8^(i+j+k+l), no noise, "
                       "RHOSVD-KRP-MEMO l=30 -> rank 20 + FP64 residual",
           "hosvd_rel_error": gold["hosvd_rel_error"]}
    for form, x in xs.items():
        ms, res = _timed(stream, lambda: K.krp_tucker_rhosvd(
            ctx, x, spec.dims, ranks, spec.oversample, spec.omega_seed, flags, core, facs),
            reps=max(3, min(args.steps, 5)), warm=2)
        esz = 4 if form == "bf16x2" else x.element_size()
        okey = "f32" if form == "f32" else "bf16"  # BF16 factors for both BF16 forms
        out[form] = {"ms": round(ms, 3), "rel_error": res["rel_residual"],
                     "oracle_rel_error": gold[f"rhosvd_memo_truncated_rel_error_{okey}"],
                     "gbs": round(3.0 * spec.numel * esz / (ms * 1e-3) / 1e9, 1)}
    out["bf16_error_over_f32"] = round(out["bf16"]["rel_error"] / out["f32"]["rel_error"], 5)
    out["bf16_speedup"] = round(out["f32"]["ms"] / out["bf16"]["ms"], 3)
    out["bf16x2_error_over_f32"] = round(out["bf16x2"]["rel_error"] / out["f32"]["rel_error"], 5)
    out["bf16x2_speedup"] = round(out["f32"]["ms"] / out["bf16x2"]["ms"], 3)
    del xs
    torch.cuda.empty_cache()
    return out


def batch_run(ctx, dev, stream, args, count=512):
    """512 uneven 3-way tensors (sides 32..192, ranks 4..16, l = r + 8):
    the batched path (one launch per phase, graph replay) in BF16 and FP32,
    against a loop of single-tensor FP32 calls."""
    import torch
    import paper_2507_23207_gb300 as K
    from synth import batch_tucker_specs
    from synth.tucker import tucker_tensor_device
    specs = batch_tucker_specs(count)
    x32, xbf = [], []
    for sp in specs:
        x64, _, _ = tucker_tensor_device(sp, device=dev)
        x32.append(x64.to(torch.float32))
        xbf.append(x64.to(torch.bfloat16))
        del x64
    torch.cuda.empty_cache()
    dims = [sp.dims for sp in specs]
    ranks = [sp.ranks for sp in specs]
    seeds = [sp.omega_seed for sp in specs]
    cores = [torch.empty(int(np.prod(sp.ranks)), dtype=torch.float32, device=dev) for sp in specs]
    facs = [[torch.empty(n * r, dtype=torch.float64, device=dev) for n, r in zip(sp.dims, sp.ranks)]
            for sp in specs]
    flags = K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL
    nelem = sum(sp.numel for sp in specs)
    out = {"workload": f"{len(specs)} tensors, sides U(32..192), ranks U(4..16), noise 1e-5, "
                       "l = r + 8, RHOSVD-KRP-MEMO + truncation + residual",
           "elements": nelem}
    reps = max(3, min(args.steps, 10))
    for form, xs, xt in (("f32", x32, K.KRP_F32), ("bf16", xbf, K.KRP_BF16)):
        items = K.make_tucker_items(xs, dims, ranks, seeds, cores, facs)
        t0 = time.perf_counter()
        rels = K.krp_tucker_rhosvd_batched(ctx, xt, items, 8, flags)  # plan, autotune, capture
        plan_s = time.perf_counter() - t0
        ms, rels = _timed(stream, lambda: K.krp_tucker_rhosvd_batched(ctx, xt, items, 8, flags),
                          reps=reps, warm=2)
        info = K.krp_tucker_batch_plan_info(ctx)
        esz = xs[0].element_size()
        out[form] = {"ms": round(ms, 3), "tensors_per_s": round(len(specs) / (ms * 1e-3), 1),
                     "gbs": round(3.0 * nelem * esz / (ms * 1e-3) / 1e9, 1),
                     "rel_error_mean": float(np.mean(rels)), "rel_error_max": float(np.max(rels)),
                     "plan_s": round(plan_s, 3), "plan": info}
    # baseline: a loop of single-tensor FP32 calls
    def loop():
        res = []
        for b, sp in enumerate(specs):
            r = K.krp_tucker_rhosvd(ctx, x32[b], sp.dims, list(sp.ranks), 8, sp.omega_seed, flags,
                                    cores[b], facs[b])
            res.append(r["rel_residual"])
        return res
    ms_loop, rl = _timed(stream, loop, reps=1, warm=1)
    out["loop_f32_single_calls"] = {"ms": round(ms_loop, 3), "rel_error_mean": float(np.mean(rl)),
                                    "rel_error_max": float(np.max(rl))}
    out["speedup_bf16_batched_vs_loop"] = round(ms_loop / out["bf16"]["ms"], 2)
    out["speedup_f32_batched_vs_loop"] = round(ms_loop / out["f32"]["ms"], 2)
    del x32, xbf
    torch.cuda.empty_cache()
    return out


def hankel_batch_run(ctx, dev, stream, args):
    """64 block Hankel matrices (state order 8..32, blocks 4x4..8x8, 32..128
    block rows, r = order, l_r = r + 8): the batched path against a loop of
    single-matrix calls, both forms."""
    import torch
    import paper_2507_23207_gb300 as K
    from synth import batch_hankel_specs, markov_parameters
    specs = batch_hankel_specs()
    host = []
    for sp in specs:
        b = markov_parameters(sp)
        host.append(np.concatenate([np.asfortranarray(b[:, :, k]).ravel(order="F")
                                    for k in range(b.shape[2])]))
    shapes = [(sp.m, sp.n, sp.s, sp.r, sp.ell_r, sp.ell_l) for sp in specs]
    seeds = [sp.omega_seed for sp in specs]
    Us = [torch.empty((sp.r, sp.m * sp.s), dtype=torch.float64, device=dev) for sp in specs]
    Vs = [torch.empty((sp.r, sp.n * sp.s), dtype=torch.float64, device=dev) for sp in specs]
    Ss = [torch.empty(sp.r, dtype=torch.float64, device=dev) for sp in specs]
    out = {"workload": f"{len(specs)} block Hankel matrices, order U(8..32), m = n U(4..8), "
                       "s U(32..128), r = order, l_r = r + 8, l_l = 1.5 l_r"}
    reps = max(3, min(args.steps, 10))
    for form, dt, bt in (("f32", torch.float32, K.KRP_F32), ("bf16", torch.bfloat16, K.KRP_BF16)):
        blocks = [torch.from_numpy(h).to(torch.float32).to(dt).to(dev) for h in host]
        items = K.make_hankel_items(blocks, shapes, seeds, Us, Ss, Vs)
        K.krp_block_hankel_batched(ctx, bt, items)
        ms, _ = _timed(stream, lambda: K.krp_block_hankel_batched(ctx, bt, items), reps=reps, warm=2)
        def loop():
            for b, sp in enumerate(specs):
                K.krp_block_hankel_lowrank(ctx, blocks[b], sp.m, sp.n, sp.s, sp.r, sp.ell_r,
                                           sp.ell_l, sp.omega_seed, Us[b], Ss[b], Vs[b])
        ms_loop, _ = _timed(stream, loop, reps=1, warm=1)
        out[form] = {"batched_ms": round(ms, 3), "loop_ms": round(ms_loop, 3),
                     "speedup": round(ms_loop / ms, 2)}
    return out


def c4_run(ctx, dev, stream, args, reps=10, warm=3):
    """1024 x 1024 block Hankel (state order 40), Alg. 6 with l_r=50, l_l=75,
    r=40, both forms; singular values against the stored FP64 oracle's."""
    import torch
    import paper_2507_23207_gb300 as K
    from synth import hankel_config_spec, markov_parameters
    spec = hankel_config_spec("c4")
    b = markov_parameters(spec)
    flat = np.concatenate([np.asfortranarray(b[:, :, k]).ravel(order="F") for k in range(b.shape[2])])
    t32 = torch.from_numpy(flat).to(torch.float32)
    blocks = {"f32": t32.to(dev), "bf16": t32.to(torch.bfloat16).to(dev)}
    ms_, ns_, r = spec.m * spec.s, spec.n * spec.s, spec.r
    U = torch.empty((r, ms_), dtype=torch.float64, device=dev)
    V = torch.empty((r, ns_), dtype=torch.float64, device=dev)
    S = torch.empty(r, dtype=torch.float64, device=dev)
    gold = _golden()["c4"]
    out = {"workload": "1024x1024 block Hankel, 128x128 blocks of 8x8, state order 40, "
                       "Alg. 6 l_r=50 l_l=75 r=40"}
    for form, bl in blocks.items():
        ms, _ = _timed(stream, lambda: K.krp_block_hankel_lowrank(
            ctx, bl, spec.m, spec.n, spec.s, r, spec.ell_r, spec.ell_l, spec.omega_seed, U, S, V),
            reps=reps, warm=warm)
        sg = S.cpu().numpy()
        so = np.asarray(gold[f"sigma_{form}"])
        out[form] = {"ms": round(ms, 4),
                     "sigma_max_abs_diff_over_sigma1": float(np.max(np.abs(sg - so)) / so[0]),
                     "oracle_rel_error_vs_input": gold[f"rel_error_vs_input_{form}"]}
        # eigensystem realization from the rank-r factors (Sec. 4.2), and the
        # distance of its eigenvalues to the system's (known by construction)
        er = torch.empty(r, dtype=torch.float64, device=dev)
        ei = torch.empty(r, dtype=torch.float64, device=dev)
        ms_era, _ = _timed(stream, lambda: K.krp_era_realize(
            ctx, bl, spec.m, spec.n, spec.s, r, U, S, V, er, ei), reps=reps, warm=warm)
        from synth.hankel import system_matrices
        eig_true = system_matrices(spec)[3]
        eg = er.cpu().numpy() + 1j * ei.cpu().numpy()
        dist = np.abs(eg[:, None] - eig_true[None, :])
        out[form]["era"] = {"ms": round(ms_era, 4),
                            "hausdorff_to_system_eigenvalues": float(max(dist.min(1).max(),
                                                                         dist.min(0).max()))}
    out["nystrom"] = nystrom_run(ctx, dev, stream, reps, warm)
    out["two_level"] = hankel2_run(ctx, dev, stream, reps, warm)
    return out


def hankel2_run(ctx, dev, stream, reps, warm):
    """Alg. 6 on a 1024 x 1024 two-level block Hankel matrix (16 x 16 blocks,
    each a 16 x 16 block Hankel matrix of 4 x 4 blocks; a two-dimensional
    exponential sum of order 20), l_r = 30, l_l = 45, r = 20; singular values
    against the explicit matrix's (LAPACK)."""
    import torch
    import paper_2507_23207_gb300 as K
    from synth import two_level_markov_parameters
    order, m, n, s1, s2, r, lr, ll = 20, 4, 4, 16, 16, 20, 30, 45
    b = two_level_markov_parameters(order, m, n, s1, s2, seed=1107)
    t32 = torch.from_numpy(np.asfortranarray(b).ravel(order="F").copy()).to(torch.float32)
    b32 = t32.numpy().astype(np.float64).reshape(b.shape, order="F")
    h = np.zeros((m * s1 * s2, n * s1 * s2))
    for i1 in range(s1):
        for j1 in range(s1):
            for i2 in range(s2):
                for j2 in range(s2):
                    r0, c0 = m * (i2 + s2 * i1), n * (j2 + s2 * j1)
                    h[r0:r0 + m, c0:c0 + n] = b32[:, :, i1 + j1, i2 + j2]
    sv = np.linalg.svd(h, compute_uv=False)[:r]
    ms, ns = m * s1 * s2, n * s1 * s2
    U = torch.empty((r, ms), dtype=torch.float64, device=dev)
    V = torch.empty((r, ns), dtype=torch.float64, device=dev)
    S = torch.empty(r, dtype=torch.float64, device=dev)
    out = {"workload": "1024x1024 two-level block Hankel (16x16 blocks of 16x16 blocks of 4x4), "
                       "order 20, l_r=30 l_l=45 r=20"}
    for form, bl in (("f32", t32.to(dev)), ("bf16", t32.to(torch.bfloat16).to(dev))):
        ms_, _ = _timed(stream, lambda: K.krp_block_hankel2_lowrank(
            ctx, bl, m, n, s1, s2, r, lr, ll, 0, U, S, V), reps=reps, warm=warm)
        out[form] = {"ms": round(ms_, 4),
                     "sigma_max_abs_diff_over_sigma1": float(np.max(np.abs(S.cpu().numpy() - sv)) / sv[0])}
    return out


def cauchy_run(ctx, dev, stream, args, n=250, ranks=(5, 10, 20, 30, 40, 50)):
    """The Tucker sweep of Sec. 5.3 on the GPU: the 4-way Cauchy tensor
    (n = 250, alpha = 2, FP32, 15.6 GB), the same target rank r in every mode
    and no oversampling, RHOSVD-KRP (fresh factors per mode), RHOSVD-KRP-MEMO
    and RSTHOSVD-KRP; the library's relative error and its phase times in the
    paper's categories (RNG, mult/KRP, QR, core; the unfolding phase is zero,
    X is never permuted).  Median of `reps` timed calls after one warm-up."""
    import torch
    import paper_2507_23207_gb300 as K
    from synth import cauchy_tensor_device
    x = cauchy_tensor_device(n, 4, 2.0, device=dev, dtype=torch.float32)
    dims = (n,) * 4
    reps = max(1, min(args.steps, 3))
    out = {"workload": f"4-way Cauchy tensor n={n}, alpha=2, FP32, l = r (no oversampling)",
           "sweep": []}
    for r in ranks:
        core = torch.empty(r ** 4, dtype=torch.float32, device=dev)
        facs = [torch.empty(n * r, dtype=torch.float64, device=dev) for _ in range(4)]
        row = {"r": r}
        for name, fn, fl in (("rhosvd_krp", K.krp_tucker_rhosvd, 0),
                             ("rhosvd_krp_memo", K.krp_tucker_rhosvd, K.KRP_MEMO),
                             ("rsthosvd_krp", K.krp_tucker_sthosvd, 0)):
            flags = fl | K.KRP_RESIDUAL | K.KRP_TIMINGS
            fn(ctx, x, dims, [r] * 4, 0, 0, flags, core, facs)
            runs = []
            for _ in range(reps):
                res = fn(ctx, x, dims, [r] * 4, 0, 0, flags, core, facs)
                runs.append(res)
            runs.sort(key=lambda z: z["times"]["total_ms"])
            med = runs[len(runs) // 2]
            t = med["times"]
            row[name] = {"ms": round(t["total_ms"], 3), "rel_error": med["rel_residual"],
                         "phases_ms": {"rng": round(t["rng_ms"], 3), "mult_krp": round(t["sketch_ms"], 3),
                                       "qr": round(t["qr_ms"], 3), "core": round(t["core_ms"], 3),
                                       "residual": round(t["residual_ms"], 3)}}
        out["sweep"].append(row)
        del core, facs
    del x
    torch.cuda.empty_cache()
    return out


def sensor_run(ctx, dev, stream, args):
    """Sensor placement (Sec. 6) at the size of the paper's flow data (not
    available; synthetic stand-in): a 150 x 90 x 60 grid with 150 training
    and 61 test snapshots of a Tucker field (core 12 x 10 x 8 x 20, noise
    1e-4, FP32).  Training: RHOSVD-KRP-MEMO of the 150 x 90 x 60 x 150
    training tensor (ranks 12, 10, 8, 20, oversampling 8), then the sensor
    grid (20 x 18 x 16) from its spatial factors; test: every test snapshot
    rebuilt from its values on the grid.  Times by CUDA events (training and
    selection: mean of three calls; reconstruction: median over the test
    snapshots), errors relative to each snapshot."""
    import torch
    import paper_2507_23207_gb300 as K
    from synth import TuckerSpec
    from synth.tucker import tucker_tensor_device
    dims, n_train = (150, 90, 60, 211), 150
    spec = TuckerSpec("snapshots", dims, (12, 10, 8, 20), 1e-4, None, 1106, (12, 10, 8, 20),
                      (20, 18, 16, 28))
    xt, _, _ = tucker_tensor_device(spec, device=dev)
    x = xt.to(torch.float32)
    del xt
    train = x[:n_train]
    tdims = dims[:3] + (n_train,)
    ells = list(spec.ell)
    core = torch.empty(int(np.prod(ells)), dtype=torch.float32, device=dev)
    facs = [torch.empty(n * c, dtype=torch.float64, device=dev) for n, c in zip(tdims, ells)]
    sp = dims[:3]
    sp_ells = ells[:3]
    idx = [torch.empty(l, dtype=torch.int32, device=dev) for l in sp_ells]
    A = [torch.empty((l, n), dtype=torch.float64, device=dev) for n, l in zip(sp, sp_ells)]

    def train_step():
        K.krp_tucker_rhosvd(ctx, train, tdims, spec.ranks, 8, 0, K.KRP_MEMO, core, facs)

    def select_step():
        K.krp_sensor_select(ctx, sp, sp_ells, facs[:3], idx, A)

    ms_train, _ = _timed(stream, train_step, reps=3, warm=2)
    ms_select, _ = _timed(stream, select_step, reps=3, warm=1)
    il = [i.long() for i in idx]
    out = torch.empty(int(np.prod(sp)), dtype=torch.float32, device=dev)
    errs, ms_rec = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for t in range(n_train, dims[3]):
        field = x[t]  # (60, 90, 150): mode-1 fastest
        t_hat = field.index_select(0, il[2]).index_select(1, il[1]).index_select(2, il[0]).contiguous()
        e0.record(stream)
        K.krp_sensor_reconstruct(ctx, sp, sp_ells, A, t_hat, out)
        e1.record(stream)
        e1.synchronize()
        ms_rec.append(e0.elapsed_time(e1))
        f = field.reshape(-1)
        errs.append(float(torch.linalg.vector_norm(out - f) / torch.linalg.vector_norm(f)))
    del x, train
    torch.cuda.empty_cache()
    return {"workload": "150x90x60 grid, 150 training + 61 test snapshots (synthetic Tucker field, "
                        "core 12x10x8x20, noise 1e-4, FP32); sensor grid 20x18x16",
            "training_rhosvd_krp_memo_ms": round(ms_train, 3), "selection_ms": round(ms_select, 3),
            "reconstruct_ms_median": round(sorted(ms_rec)[len(ms_rec) // 2], 4),
            "test_rel_error_mean": float(np.mean(errs)), "test_rel_error_max": float(np.max(errs))}


def hadamard_run(ctx, dev, stream, args):
    """Recompression of the Hadamard product of two Tucker tensors (Sec. 5):
    512^3 tensors with Tucker ranks 8 (the product has rank 64 per mode),
    l = 24.  Structured path (krp_tucker_hadamard, FP64, the product never
    formed) against forming the 512^3 product on the device (FP32) and running
    krp_tucker_rhosvd (MEMO) on it.  CUDA events, mean of three calls after
    a warm-up; both errors as the library reports them."""
    import torch
    import paper_2507_23207_gb300 as K
    from synth import haar
    dims, r, ell = (512, 512, 512), (8, 8, 8), 24
    rng = np.random.default_rng(1108)
    g = rng.standard_normal(r)
    h = rng.standard_normal(r)
    us = [haar(n, k, rng) for n, k in zip(dims, r)]
    vs = [haar(n, k, rng) for n, k in zip(dims, r)]
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a.T)).to(dev)
    G = torch.from_numpy(np.ascontiguousarray(g.T)).to(dev)
    H = torch.from_numpy(np.ascontiguousarray(h.T)).to(dev)
    U = [to(u) for u in us]
    V = [to(v) for v in vs]
    core = torch.empty(ell ** 3, dtype=torch.float64, device=dev)
    facs = [torch.empty((ell, n), dtype=torch.float64, device=dev) for n in dims]
    out = {"workload": "Hadamard product of two 512^3 Tucker tensors of rank 8 (product rank 64), l = 24"}
    err = [0.0]

    def structured():
        err[0] = K.krp_tucker_hadamard(ctx, dims, r, G, U, r, H, V, ell, 0, core, facs)

    ms, _ = _timed(stream, structured, reps=3, warm=1)
    out["structured_fp64"] = {"ms": round(ms, 4), "rel_error": err[0]}

    def explicit():
        # X, Y in torch layout (n3, n2, n1) from the FP64 cores and factors
        x = torch.einsum("cba,ic,jb,ka->ijk", G, U[2].T, U[1].T, U[0].T)
        y = torch.einsum("cba,ic,jb,ka->ijk", H, V[2].T, V[1].T, V[0].T)
        z = (x * y).to(torch.float32).contiguous()
        c32 = torch.empty(ell ** 3, dtype=torch.float32, device=dev)
        f64 = [torch.empty(n * ell, dtype=torch.float64, device=dev) for n in dims]
        res = K.krp_tucker_rhosvd(ctx, z, dims, [ell] * 3, 0, 0, K.KRP_MEMO | K.KRP_RESIDUAL, c32, f64)
        err[0] = res["rel_residual"]

    ms, _ = _timed(stream, explicit, reps=3, warm=1)
    out["explicit_product_fp32"] = {"ms": round(ms, 4), "rel_error": err[0],
                                    "note": "forms X, Y and Z = X * Y on the device, then RHOSVD-KRP-MEMO"}
    return out


def nystrom_run(ctx, dev, stream, reps, warm):
    """Nystrom approximation (the remark after Alg. 6) of a symmetric positive
    semidefinite block Hankel matrix of the same size (symmetric system of
    order 40, 128 x 128 blocks of 8 x 8), l = 50, r = 40, default cut-off;
    eigenvalues against the input's (LAPACK on the explicit 1024 x 1024)."""
    import torch
    import paper_2507_23207_gb300 as K
    from synth import HankelSpec, symmetric_markov_parameters
    spec = HankelSpec("spsd", 40, 8, 8, 128, 0.95, 1104, 40, 50, 50)
    b = symmetric_markov_parameters(spec)
    flat = np.concatenate([np.asfortranarray(b[:, :, k]).ravel(order="F") for k in range(b.shape[2])])
    t32 = torch.from_numpy(flat).to(torch.float32)
    ms_, r, ell = spec.m * spec.s, 20, spec.ell_r
    s = spec.s
    h = np.zeros((ms_, ms_))
    bb = t32.numpy().astype(np.float64).reshape(2 * s - 1, 8, 8)
    for i in range(s):
        for j in range(s):
            h[i * 8:(i + 1) * 8, j * 8:(j + 1) * 8] = bb[i + j].T
    lam_in = np.sort(np.linalg.eigvalsh(h))[::-1][:r]
    U = torch.empty((r, ms_), dtype=torch.float64, device=dev)
    L = torch.empty(r, dtype=torch.float64, device=dev)
    out = {"workload": "1024x1024 SPSD block Hankel (symmetric system, order 40), 128x128 "
                       "blocks of 8x8, l=50, top r=20 eigenpairs, cut-off 1e-5"}
    for form, bl in (("f32", t32.to(dev)), ("bf16", t32.to(torch.bfloat16).to(dev))):
        ms, _ = _timed(stream, lambda: K.krp_block_hankel_nystrom(ctx, bl, 8, s, r, ell, 0, U, L),
                       reps=reps, warm=warm)
        lg = L.cpu().numpy()
        out[form] = {"ms": round(ms, 4),
                     "eig_max_abs_diff_over_lambda1": float(np.max(np.abs(lg - lam_in)) / lam_in[0])}
    return out


# DRAM traffic (read + write bytes) per launch at 1024^3, from ncu captures at
# 512^3 (dram__bytes_read.sum + dram__bytes_write.sum) scaled by the bytes
# each part moves: X x8; the TTM's output (S x l) x4; the residual's H hi/lo
# rows (S x 64) x4; the per-CTA atomic adds of the MTTKRP and the residual
# (one row block of Y_1, two sums per CTA) x1.  A kernel changed since its
# capture has no entry (null in the line).
TRAFFIC_1024 = {
    "tc_gemm_tn_tf32": 537.192192e6 * 8 + 43.580416e6 * 4,
    "tc_mttkrp_tf32": 537.426176e6 * 8 + 3.841792e6,
    "tc_residual_tf32": 537.2e6 * 8 + (604.1536e6 - 537.2e6) * 4 + 3.219456e6,
}


def _kernel_work(name, spec):
    """(kernel, bound, unit, algorithmic work per launch) of the kernels of the
    FP32 step that can dominate it, at the launch size that reads all of X."""
    n, ell = spec.numel, max(spec.ell)
    r = min(spec.ranks)
    s1 = n / spec.dims[0]
    if name == "tc_mttkrp_tf32":
        return ("tc_mttkrp_tf32_kernel (FP32 mode-1 sketch Y_1 = X_(1)(Omega_3 kr Omega_2) on "
                "tcgen05, three TF32 products)", "hbm", "GB/s", n * 4.0 + spec.dims[0] * ell * 4.0)
    if name == "tc_gemm_tn_tf32":
        return ("tc_gemm_tn_tf32_kernel (FP32 TTM X_(1)^T F on tcgen05, three TF32 products)",
                "hbm", "GB/s", n * 4.0 + s1 * ell * 4.0)
    if name == "tc_residual_tf32":
        return ("tc_residual_tf32_kernel (FP32 residual ||X - Q_1 H|| on tcgen05, three TF32 "
                "products)", "hbm", "GB/s", n * 4.0 + s1 * r * 8.0)
    if name == "krp_slab_mttkrp_f32":
        return ("krp_slab_mttkrp_kernel<48> (FP32 mode-1 sketch, FFMA)", "alu", "TFLOP/s",
                2.0 * n * ell)
    if name == "residual":
        return ("residual_tiled_kernel (FP32 residual ||X - Q_1 H||, FFMA)", "alu", "TFLOP/s",
                2.0 * n * r)
    return None


def _big_launches(times, steps):
    """The launches of one kernel name that read all of X: the largest
    (launches per step that take at least half the largest one's time) x steps."""
    per = max(1, len(times) // max(1, steps))
    top = max(times)
    big = sorted(times)[-per * steps:]
    return [t for t in big if t >= 0.5 * top]


def trace_roofline(spec, f32, peaks, args):
    """Roofline of the dominant kernel of the FP32 step: the kernel with the
    largest share of the step in the launch trace (CUDA events after every
    launch on the context stream over the timed steps), among the mode-1
    MTTKRP, the TTM over X (two launches per step: the tree's B-part and the
    core's first TTM) and the residual.  `achieved` = its algorithmic work
    per launch / its average launch time; the other candidates are reported
    beside it."""
    tr = f32.get("trace") or []
    # the timed step (launches on the second stream overlap the first's)
    step_ms = f32.get("ms") or sum(t for _, t in tr) / max(1, args.steps)
    tot = {}
    for name, t in tr:
        if _kernel_work(name, spec):
            tot.setdefault(name, []).append(t)
    if not tot or step_ms <= 0:
        return {"error": "no traced kernel of the FP32 step"}
    mhz = (f32.get("clocks") or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    sms = sm_count()

    def one(name):
        label, bound, unit, work = _kernel_work(name, spec)
        times = _big_launches(tot[name], args.steps)
        t_avg = sum(times) / len(times)
        if bound == "alu":
            peak = fp32_ffma_peak_tflops(mhz, sms)
            ach = work / (t_avg * 1e-3) / 1e12
            note = f"FP32 FFMA peak = {sms} SMs x 128 lanes x 2 flop x {mhz:.0f} MHz"
        else:
            peak = peaks["hbm_gbs"]
            ach = work / (t_avg * 1e-3) / 1e9
            note = "hbm_gbs of MEASURED_PEAKS.json"
        return {"kernel": label, "bound": bound, "achieved": round(ach, 3), "peak": round(peak, 3),
                "unit": unit, "frac": round(ach / peak, 4), "traffic": TRAFFIC_1024.get(name),
                "ms_per_launch": round(t_avg, 4), "launches_averaged": len(times),
                "kernel_share_of_step": round(sum(tot[name]) / args.steps / step_ms, 4),
                "peak_note": note}

    name = max(tot, key=lambda k: sum(tot[k]))
    out = one(name)
    out["timing"] = "CUDA events after every launch on the context stream over the timed steps"
    out["beside"] = {k: one(k) for k in sorted(tot) if k != name}
    return out


def sketch_rooflines(ctx, spec, forms, dev, stream, peaks, clk, args):
    """The all-mode KRP sketch alone (krp_sketch_all_modes with the memoized
    factor set, Sec. 5.1) in each form, against one pass over X at the
    measured HBM bandwidth: the FP32 form as the mode-1 MTTKRP and the TTM
    X_(1)^T Omega_1 (two passes, both on tensor cores as TF32 products), the
    BF16 and BF16 hi/lo forms as the one-pass tree (their 4 N l flops need
    well under the tensor peak).  The kernels of one call and their times
    come from the launch trace."""
    import torch
    import paper_2507_23207_gb300 as K
    ell = max(spec.ell)
    n = spec.numel
    mhz = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    sms = sm_count()
    ffma = fp32_ffma_peak_tflops(mhz, sms)
    hbm = float(peaks["hbm_gbs"])
    reps = max(5, args.steps)
    out = {"workload": f"krp_sketch_all_modes, {'x'.join(map(str, spec.dims))}, l = {ell}, "
                       "memoized factor set (one pass over X for the tensor-core forms)",
           "timing": f"CUDA events over {reps} calls after 3 warm-ups; kernel times from the "
                     "launch trace (an event after every launch) over 3 more calls"}
    for form, x in forms:
        dt = torch.float32 if form == "f32" else torch.bfloat16
        om = [torch.empty((ell, m), dtype=dt, device=dev) for m in spec.dims]
        K.krp_gen_factors(ctx, spec.omega_seed, K.KRP_DRAW_MEMO, K.KRP_TAG_OMEGA, spec.dims, ell, om)
        ys = [torch.empty((ell, m), dtype=torch.float32, device=dev) for m in spec.dims]
        ms, _ = _timed(stream, lambda: K.krp_sketch_all_modes(ctx, x, spec.dims, om, ell, ys),
                       reps=reps, warm=3)
        K.krp_trace_begin(ctx)
        for _ in range(3):
            K.krp_sketch_all_modes(ctx, x, spec.dims, om, ell, ys)
        tr = K.krp_trace_end(ctx)
        agg = {}
        for nm, t in tr:
            agg[nm] = agg.get(nm, 0.0) + t / 3
        top = max(agg, key=agg.get)
        b = 4 if form in ("f32", "bf16x2") else 2
        gbs = n * b / (ms * 1e-3) / 1e9
        tfl = 4.0 * n * ell / (ms * 1e-3) / 1e12
        e = {"ms": round(ms, 4), "gbs": round(gbs, 1), "tflops": round(tfl, 2),
             "bytes_per_elem": b, "kernels_ms": {k: round(v, 4) for k, v in
                                                 sorted(agg.items(), key=lambda kv: -kv[1])}}
        t_top = agg[top]
        if form == "f32" and "tc_mttkrp_tf32" in agg:
            # the FP32 form's tree takes two passes over X (the mode-1 MTTKRP,
            # then the TTM X_(1)^T Omega_1), both on tensor cores; the
            # algorithmic minimum is one pass at the measured HBM bandwidth
            t_min = n * 4.0 / (hbm * 1e9) * 1e3
            e["roofline"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm,
                             "unit": "GB/s", "frac": round(gbs / hbm, 4),
                             "t_min_ms": round(t_min, 4), "passes_over_x": 2,
                             "peak_note": "hbm_gbs of MEASURED_PEAKS.json; achieved = 4 N bytes "
                                          "(one pass) / the call's time"}
            e["dominant_kernel"] = {"name": top, "ms": round(t_top, 4),
                                    "gbs": round(n * b / (t_top * 1e-3) / 1e9, 1),
                                    "frac": round(n * b / (t_top * 1e-3) / 1e9 / hbm, 4)}
        elif form == "f32":
            e["roofline"] = {"bound": "alu", "achieved": round(tfl, 3), "peak": round(ffma, 3),
                             "unit": "TFLOP/s", "frac": round(tfl / ffma, 4),
                             "peak_note": f"FP32 FFMA peak = {sms} SMs x 128 lanes x 2 flop x "
                                          f"{mhz:.0f} MHz (derived)"}
        else:
            e["roofline"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm,
                             "unit": "GB/s", "frac": round(gbs / hbm, 4),
                             "peak_note": "hbm_gbs of MEASURED_PEAKS.json"}
            e["dominant_kernel"] = {"name": top, "ms": round(t_top, 4),
                                    "gbs": round(n * b / (t_top * 1e-3) / 1e9, 1),
                                    "frac": round(n * b / (t_top * 1e-3) / 1e9 / hbm, 4)}
        out[form] = e
        del om, ys
    return out


def e2e_run(ctx, spec, x32, args):
    import torch
    import paper_2507_23207_gb300 as K
    host = torch.empty(x32.shape, dtype=torch.float32, pin_memory=True)
    host.copy_(x32)
    ranks = list(spec.ranks)
    core = torch.empty(int(np.prod(ranks)), dtype=torch.float32, pin_memory=True)
    facs = [torch.empty(n * r, dtype=torch.float64, pin_memory=True) for n, r in zip(spec.dims, ranks)]
    flags = K.KRP_MEMO | K.KRP_TRUNCATE | K.KRP_RESIDUAL
    K.krp_tucker_rhosvd(ctx, host, spec.dims, ranks, spec.oversample, spec.omega_seed, flags, core, facs)
    torch.cuda.synchronize()
    # host-timed steps; the median, since a step now and then stalls on the
    # shared host (seen: one step of 49 ms or 133 ms among steps of 23.6 ms)
    reps = max(3, min(args.steps, 7))
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        res = K.krp_tucker_rhosvd(ctx, host, spec.dims, ranks, spec.oversample, spec.omega_seed,
                                  flags, core, facs)
        torch.cuda.synchronize()
        times.append((time.perf_counter() - t0) * 1e3)
    ms = float(np.median(times))
    mean_ms = float(np.mean(times))
    d2h = core.numel() * 4 + sum(f.numel() * 8 for f in facs) + 8
    # the host-to-device copy of X alone, for comparison (CUDA events)
    dst = torch.empty_like(x32)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    dst.copy_(host, non_blocking=True)
    copies = []
    for _ in range(3):  # median of three (the shared host stalls a copy now and then)
        e0.record()
        dst.copy_(host, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        copies.append(e0.elapsed_time(e1))
    h2d_ms = float(np.median(copies))
    del dst
    return {"ms": ms, "mean_ms": mean_ms, "reps": reps, "h2d": spec.numel * 4, "d2h": d2h,
            "resid": res["rel_residual"], "h2d_ms": h2d_ms}


def _oracle_sample(spec, k):
    """One oracle run (RHOSVD-KRP-MEMO + truncation + explicit residual, in
    the order of oracle.tucker.rhosvd_krp) on the slab X[:, :, :k], timed per
    phase in the paper's categories (RNG, mult/KRP, QR, core) plus truncation
    and residual.  Returns (phase seconds, total seconds, entries)."""
    from oracle import linalg as LA, philox, tensor as T, tucker as TK
    from synth.tucker import expand_tucker, tucker_factors
    g0, us = tucker_factors(spec)
    us_k = list(us)
    us_k[-1] = us[-1][:k]
    xs = philox.round_to_f32(expand_tucker(g0, us_k))
    ells = list(spec.ell)
    ph = {}
    t0 = time.perf_counter()
    shared = TK.memo_factors(spec.omega_seed, xs.shape, max(ells), "f32")
    t1 = time.perf_counter()
    ys = [T.mttkrp(xs, [f[:, :ells[i]] if j != i else None for j, f in enumerate(shared)], i)
          for i in range(xs.ndim)]
    t2 = time.perf_counter()
    qs = [LA.householder_qr(y)[0] for y in ys]
    t3 = time.perf_counter()
    g = T.multi_ttm(xs, [q.T for q in qs])
    t4 = time.perf_counter()
    g2, q2 = TK.truncate_core(g, qs, list(spec.ranks))
    t5 = time.perf_counter()
    TK.rel_error(xs, g2, q2)
    t6 = time.perf_counter()
    ph = {"rng_s": t1 - t0, "mult_krp_s": t2 - t1, "qr_s": t3 - t2, "core_s": t4 - t3,
          "truncate_s": t5 - t4, "residual_s": t6 - t5}
    return ph, t6 - t0, xs.size


def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _sample_in_subprocess(spec_args, k, threads):
    """The oracle sample in a fresh process (no CUDA state), with the BLAS and
    OpenMP thread counts fixed before numpy loads (threads None = all cores)."""
    env = dict(os.environ)
    if threads is not None:
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                  "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS"):
            env[v] = str(threads)
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", str(k)] + spec_args
    res = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if res.returncode != 0:
        raise RuntimeError(res.stderr[-500:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def cpu_baseline(spec, spec_args, target_s=10.0, k=None, threads=None):
    """The FP64 oracle (RHOSVD-KRP-MEMO + truncation + explicit residual) on a
    slab sample X[:, :, :k] of the same workload, timed on the host cores
    (threads None: all of them; 1: a single thread) with per-phase times.
    Without k, the slab depth doubles from max(l) until one sample takes at
    least target_s seconds (or the slab is the whole tensor), and that sample
    is reported."""
    if k is None:
        k = max(spec.ell)  # the slab depth must allow l_d columns in the last mode
        while True:
            r = _sample_in_subprocess(spec_args, k, threads)
            if r["seconds"] >= target_s or k >= spec.dims[-1]:
                break
            k = min(spec.dims[-1], 2 * k)
    else:
        r = _sample_in_subprocess(spec_args, k, threads)
    dt, n = r["seconds"], r["entries"]
    gbs = 3 * n * 4 / dt / 1e9
    cores = threads if threads is not None else (os.cpu_count() or 1)
    return {"value": round(gbs, 4), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "cpu_model": _cpu_model(),
            "sample": f"slab sample X[:, :, :{k}] of {spec.name} ({n} entries), one "
                      f"RHOSVD-KRP-MEMO + truncation + explicit residual, {dt:.2f} s",
            "seconds": round(dt, 3), "slab_depth": k,
            "phases_s": {p: round(v, 3) for p, v in r["phases"].items()}}


def run_sharded(args, rank, world, local_rank):
    """RHOSVD-KRP-MEMO of the one workload tensor split into slabs of its last
    mode, one per rank (paper_2507_23207_gb300.sharded): every rank runs the
    C-ABI steps on its slab and the ranks all-reduce the packed sketches, the
    core and the residual sums (NCCL under torchrun; at N = 1 the reductions
    are the identity).  Total work is fixed as N grows (strong scaling)."""
    import torch
    import paper_2507_23207_gb300 as K
    from paper_2507_23207_gb300.sharded import CudaOps, exchange_bytes, rhosvd_sharded, slab_bounds
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    spec = workload(args)
    x32, _ = make_inputs(spec, dev, want_bf16=False)
    start, stop = slab_bounds(spec.dims[-1], world, rank)
    xs = x32[start:stop].contiguous()  # torch layout (n_d, ..., n_1): the slab of the last mode
    del x32
    torch.cuda.empty_cache()
    ctx = K.Context(local_rank, torch.cuda.current_stream(dev).cuda_stream)
    ops = CudaOps(ctx, dev)
    red = None if world > 1 else (lambda t: None)

    def step():
        return rhosvd_sharded(ops, xs, spec.dims, start, stop, list(spec.ranks), spec.oversample,
                              spec.omega_seed, allreduce=red)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        core, qs, rel = step()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    ctx.close()
    if rank != 0:
        return
    n = spec.numel
    line = {"metric": METRIC, "value": round(3.0 * n * 4 / (ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{spec.name}: {'x'.join(map(str, spec.dims))} FP32, "
                       f"RHOSVD-KRP-MEMO + truncation + residual, one slab of the last mode per rank",
                       "parallelism": f"slab-sharded x{world}",
                       "l2": "inputs larger than L2 (no flush)"},
            "rel_error": rel,
            "allreduce_bytes_per_rank_per_step": exchange_bytes(spec.dims, spec.ranks,
                                                                spec.oversample),
            "note": "per-rank C-ABI steps (factors, sketch, QR, multi-TTM, truncation, residual) "
                    "with NCCL all-reduces between them"}
    print(json.dumps(line))


def workload(args):
    from dataclasses import replace
    from synth import config_spec
    spec = config_spec(args.config)
    if args.dims:
        dims = tuple(int(v) for v in args.dims.split(","))
        spec = replace(spec, name=spec.name + "@" + "x".join(map(str, dims)), dims=dims)
    return spec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--dims", default=None,
                    help="override the tensor sides (comma separated), e.g. for profiling")
    ap.add_argument("--no-bf16", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the STHOSVD, 200^4 and block-Hankel measurements")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched workloads (for profiling) and print their line")
    ap.add_argument("--batch-count", type=int, default=512,
                    help="tensors in the batched workload with --batch-only")
    ap.add_argument("--hadamard", action="store_true",
                    help="run only the Hadamard-product recompression workload and print its line")
    ap.add_argument("--sensor", action="store_true",
                    help="run only the sensor-placement workload and print its line")
    ap.add_argument("--cauchy", action="store_true",
                    help="run only the Cauchy-tensor Tucker sweep (4-way, n = 250) and print its line")
    ap.add_argument("--hankel-only", action="store_true",
                    help="run only the 1024 x 1024 block-Hankel measurement (for profiling)")
    ap.add_argument("--sketch-only", action="store_true",
                    help="run only the all-mode sketch of each form (for profiling) and print it")
    ap.add_argument("--forms", default="f32,bf16,bf16x2",
                    help="forms of --sketch-only (comma separated)")
    ap.add_argument("--sharded", action="store_true",
                    help="split the tensor into slabs of its last mode, one per rank, with "
                         "all-reduces between the steps (strong scaling)")
    ap.add_argument("--cpu-sample", type=int, default=None,
                    help="(internal) time one oracle sample of slab depth K and print it")
    args = ap.parse_args()
    spec_args = ["--config", args.config] + (["--dims", args.dims] if args.dims else [])

    if args.cpu_sample is not None:
        ph, dt, n = _oracle_sample(workload(args), args.cpu_sample)
        print(json.dumps({"phases": ph, "seconds": dt, "entries": n}))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        spec = workload(args)
        # the slab depth is chosen once (that search is the first warm-up),
        # then every step times the oracle on the same slab
        k = cpu_baseline(spec, spec_args, target_s=4.0)["slab_depth"]
        for _ in range(args.warmup - 1):
            cpu_baseline(spec, spec_args, k=k)
        vals = [cpu_baseline(spec, spec_args, k=k) for _ in range(max(1, args.steps))]
        v = float(np.median([c["value"] for c in vals]))
        line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1e3 * float(np.median([c["seconds"] for c in vals])), 2),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": spec.name + " slab sample"},
                "cpu_baseline": {f: vals[-1][f] for f in ("kind", "cores", "sample", "cpu_model",
                                                          "phases_s")} | {"value": round(v, 4)},
                "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if args.hadamard:
        import torch
        import paper_2507_23207_gb300 as K
        dev = torch.device(f"cuda:{local_rank}")
        torch.cuda.set_device(dev)
        stream = torch.cuda.current_stream(dev)
        ctx = K.Context(local_rank, stream.cuda_stream)
        out = {"hadamard_512cubed": hadamard_run(ctx, dev, stream, args)}
        ctx.close()
        print(json.dumps(out))
        return

    if args.sensor:
        import torch
        import paper_2507_23207_gb300 as K
        dev = torch.device(f"cuda:{local_rank}")
        torch.cuda.set_device(dev)
        stream = torch.cuda.current_stream(dev)
        ctx = K.Context(local_rank, stream.cuda_stream)
        out = {"sensor_placement": sensor_run(ctx, dev, stream, args)}
        ctx.close()
        print(json.dumps(out))
        return

    if args.cauchy:
        import torch
        import paper_2507_23207_gb300 as K
        dev = torch.device(f"cuda:{local_rank}")
        torch.cuda.set_device(dev)
        stream = torch.cuda.current_stream(dev)
        ctx = K.Context(local_rank, stream.cuda_stream)
        out = {"cauchy_250": cauchy_run(ctx, dev, stream, args)}
        ctx.close()
        print(json.dumps(out))
        return

    if args.hankel_only:
        import torch
        import paper_2507_23207_gb300 as K
        dev = torch.device(f"cuda:{local_rank}")
        torch.cuda.set_device(dev)
        stream = torch.cuda.current_stream(dev)
        ctx = K.Context(local_rank, stream.cuda_stream)
        out = {"block_hankel_1024": c4_run(ctx, dev, stream, args, reps=max(1, args.steps),
                                           warm=max(1, args.warmup))}
        ctx.close()
        print(json.dumps(out))
        return

    if args.sketch_only:
        import torch
        import paper_2507_23207_gb300 as K
        dev = torch.device(f"cuda:{local_rank}")
        torch.cuda.set_device(dev)
        stream = torch.cuda.current_stream(dev)
        spec = workload(args)
        want = set(args.forms.split(","))
        x32, xbf = make_inputs(spec, dev, want_bf16="bf16" in want)
        ctx = K.Context(local_rank, stream.cuda_stream)
        forms = []
        if "f32" in want:
            forms.append(("f32", x32))
        if "bf16" in want:
            forms.append(("bf16", xbf))
        if "bf16x2" in want:
            forms.append(("bf16x2", K.krp_split_bf16x2(ctx, x32)))
        peaks, _ = measured_peaks()
        out = sketch_rooflines(ctx, spec, forms, dev, stream, peaks, None, args)
        ctx.close()
        print(json.dumps({"sketch": out}))
        return

    if args.batch_only:
        import torch
        import paper_2507_23207_gb300 as K
        dev = torch.device(f"cuda:{local_rank}")
        torch.cuda.set_device(dev)
        stream = torch.cuda.current_stream(dev)
        ctx = K.Context(local_rank, stream.cuda_stream)
        out = {"batched_tucker": batch_run(ctx, dev, stream, args, count=args.batch_count),
               "batched_hankel": hankel_batch_run(ctx, dev, stream, args)}
        ctx.close()
        print(json.dumps(out))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.sharded:
        run_sharded(args, rank, world, local_rank)
        return
    spec, results, kr, sketch, e2e, peaks, peak_src, (sk, co, rs, qr), extra = run_ours(
        args, rank, world, local_rank)
    if rank != 0:
        return
    f32 = results["f32"]
    n = spec.numel
    bytes_step = 3.0 * n * 4
    flops_step = sk + co + rs + qr
    ms = f32["ms"]
    value = world * bytes_step / (ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu and world == 1:   # the host baseline is timed at N = 1 only
        try:
            cpu = cpu_baseline(spec, spec_args)
            one = cpu_baseline(spec, spec_args, target_s=5.0, threads=1)
            cpu["one_thread"] = {f: one[f] for f in ("value", "cores", "sample", "seconds",
                                                     "phases_s")}
        except Exception as exc:  # the GPU line is still printed
            cpu = {"error": repr(exc)[:300]}
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{spec.name}: {'x'.join(map(str, spec.dims))} FP32, multilinear rank "
                   f"{spec.core[0]} + {spec.noise:g} noise, l={spec.ell[0]}, r={spec.ranks[0]}, "
                   "RHOSVD-KRP-MEMO + FP64 QR + core + FP64 truncation + FP64 residual",
                   "l2": "inputs larger than L2 (no flush)", "replicas": world},
        "tflops": round(world * flops_step / (ms * 1e-3) / 1e12, 3),
        "rhosvd_ms": round(ms, 3),
        "rel_error": f32["res"]["rel_residual"],
        "phases_ms": {k: round(v, 4) for k, v in f32["phases"].items()},
        "clocks": f32["clocks"],
        "gpu_launches": f32["launches"],
        "roofline": kr,
        "sketch": sketch,
        "peaks_source": peak_src,
    }
    if "bf16" in results:
        b = results["bf16"]
        line["bf16_form"] = {
            "ms_per_step": round(b["ms"], 4),
            "value": round(world * 3.0 * n * 2 / (b["ms"] * 1e-3) / 1e9, 2), "unit": "GB/s",
            "tflops": round(world * flops_step / (b["ms"] * 1e-3) / 1e12, 3),
            "rel_error": b["res"]["rel_residual"],
            "phases_ms": {k: round(v, 4) for k, v in b["phases"].items()},
            "speedup_vs_f32": round(ms / b["ms"], 3)}
    if "bf16x2" in results:
        b = results["bf16x2"]
        line["bf16x2_form"] = {
            "note": "X as a BF16 hi/lo pair on tensor cores (4 B per element)",
            "ms_per_step": round(b["ms"], 4),
            "value": round(world * 3.0 * n * 4 / (b["ms"] * 1e-3) / 1e9, 2), "unit": "GB/s",
            "rel_error": b["res"]["rel_residual"],
            "error_over_f32": round(b["res"]["rel_residual"] / f32["res"]["rel_residual"], 5),
            "phases_ms": {k: round(v, 4) for k, v in b["phases"].items()},
            "speedup_vs_f32": round(ms / b["ms"], 3)}
    if e2e:
        line["e2e"] = {"value": round(bytes_step / (e2e["ms"] * 1e-3) / 1e9, 2), "unit": "GB/s",
                       "ms_per_step": round(e2e["ms"], 3),
                       "timing": f"median of {e2e['reps']} host-timed steps (mean "
                                 f"{e2e['mean_ms']:.3f} ms)",
                       "h2d_bytes_per_step": e2e["h2d"],
                       "d2h_bytes_per_step": e2e["d2h"],
                       "h2d_alone_ms": round(e2e["h2d_ms"], 3),
                       "h2d_gbs": round(e2e["h2d"] / (e2e["h2d_ms"] * 1e-3) / 1e9, 1),
                       "note": "X copied in 8 chunks of the last mode on a second stream, each "
                               "chunk sketched as it lands; then QR, core, truncation, residual"}
    if cpu:
        line["cpu_baseline"] = cpu
    line.update(extra)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
