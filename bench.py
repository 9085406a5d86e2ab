#!/usr/bin/env python
"""Throughput of sound reachable-set bounds: domain-steps per second on one B300.

A step is one pass of the whole bound computation over one batch of domains: every domain's
Taylor-model seed, the per-layer back-substitution chains (3xTF32 on the tcgen05 tensor cores) and
concretisations, the controller Taylor model, the dynamics, the FP64 boxes of every horizon step and
the hull over domains.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (default): the large workload, 16-state stable linear dynamics with the ReLU controller
16-512-512-512-512-8 (FP32 weights), horizon 50, chord slopes; a step bounds a chunk of 16,384 of its
262,144 sub-boxes (rank r of N takes the r-th chunk).  Prints one JSON line on rank 0.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_25346_b300 import workloads as wl  # noqa: E402

METRIC = "sound-bound domain-steps/s (1e-5 rel vs FP64 oracle)"
UNIT = "domain-steps/s"
L2_BYTES = 126 * 2 ** 20
FP32_LANES_PER_SM = 128
SMS = 148


# DRAM bytes (read + write) of one fused forward launch on the 4096-box workload, measured with ncu
# (dram__bytes_read.sum + dram__bytes_write.sum of one steady-state launch); the working set lives in
# shared memory, so this is the boxes and weights read once.
FUSED_TRAFFIC_BYTES = 548864

# DRAM bytes (read + write) per stacked row of one persistent GEMM launch (K = N = 512):
# dram__bytes_read.sum + dram__bytes_write.sum of one launch over R = 65,536 rows (ncu, small case),
# divided by R.  The traffic grows with R (the left operand is read once; the chain level also writes
# the next one once), so a full launch's traffic is this times its rows.
GEMM_TRAFFIC_PER_ROW = {"final": (271.55e6 + 19.45e6) / 65536, "chain": (271.54e6 + 226.41e6) / 65536}
# launches of at least this many stacked rows are the full-size ones (hidden-layer targets:
# domains x 512 rows); the controller-output target's launches have domains x 8 rows
BIG_GEMM_ROWS = 65536

HEADLINE_CHUNK = 16384


def fused_flops_per_domain_step(widths):
    """Algorithmic FLOPs (2 per multiply-add) of one domain-step of the forward pass.

    Per target layer l: chain levels m = l-1..1 cost n_l*n_m*(3 + n_{m-1}) MACs (intercepts
    Lambda^+ d, Lambda^- d, Lambda_s b and the product Lambda_s W_m); the concretisation costs
    n_l*n*(n + 3) MACs (Lambda P, Lambda c, the remainder interval); the dynamics cost
    n*(n+m)*(n + 3) MACs (P', c', I').
    """
    n, m, L = widths[0], widths[-1], len(widths) - 1
    mac = 0
    for l in range(1, L + 1):
        for mm in range(l - 1, 0, -1):
            mac += widths[l] * widths[mm] * (3 + widths[mm - 1])
        mac += widths[l] * n * (n + 3)
    mac += n * (n + m) * (n + 3)
    return 2 * mac


def measure_refinement(local):
    """Slope refinement on the cart-pole workload (1024 sub-boxes, H=20, 20 projected-gradient steps):
    batched over all domains vs the plain per-domain form (one domain per call) on a sample."""
    from paper_2605_25346_b300 import api
    p = wl.cartpole_diff()
    r = api.Reach(local).load(p)
    r.optimize(1, 0.1, 0.0)  # warm-up (also compiles/loads every kernel)
    r.close()
    r = api.Reach(local).load(p)
    torch.cuda.synchronize()
    l0 = r.launches()
    t0 = time.perf_counter()
    hist = r.optimize(p.alpha_steps, 0.1, 0.0)
    tb = time.perf_counter() - t0
    launches = r.launches() - l0
    Vb = r.objective()
    r.close()
    sample = 8
    tp, Vp = 0.0, []
    for d in range(sample):
        q = p.subset([d])
        rr = api.Reach(local).load(q)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rr.optimize(p.alpha_steps, 0.1, 0.0)
        tp += time.perf_counter() - t0
        Vp.append(rr.objective()[0])
        rr.close()
    gap = float(np.max(np.abs(np.array(Vp) - Vb[:sample]) / np.abs(Vb[:sample])))
    out = {"workload": "cart-pole 4-128-128-2, 1024 sub-boxes, H=20, 20 steps, lr 0.1",
           "alpha_opt_steps_per_s": p.alpha_steps / tb, "batched_domains_per_s": p.D / tb,
           "plain_domains_per_s": sample / tp, "plain_sample_domains": sample,
           "batched_over_plain": (p.D / tb) / (sample / tp), "max_rel_V_gap_batched_vs_plain": gap,
           "V_first": float(hist[0]), "V_best": float(hist[-1]),
           "V_reduction": 1.0 - float(hist[-1]) / float(hist[0]), "gpu_launches": int(launches)}
    # the same from slopes 0.05 off the chord point, where refinement changes V substantially (the
    # chord point is a local minimum of V): batched vs plain at that refined gap
    r = api.Reach(local).load(p)
    a0 = r.get_alpha()
    start = np.where(a0 > 0, np.clip(a0 + 0.05, 0.0, 1.0), a0).astype(np.float32)
    r.set_alpha(start)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = r.optimize(p.alpha_steps, 0.1, 0.0)
    tb = time.perf_counter() - t0
    Vb = r.objective()
    r.close()
    tp, Vp = 0.0, []
    for d in range(sample):
        rr = api.Reach(local).load(p.subset([d]))
        rr.set_alpha(start[d:d + 1])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rr.optimize(p.alpha_steps, 0.1, 0.0)
        tp += time.perf_counter() - t0
        Vp.append(rr.objective()[0])
        rr.close()
    out["from_perturbed_start"] = {
        "start": "chord slopes + 0.05 on unstable neurons", "V_first": float(hist[0]), "V_best": float(hist[-1]),
        "V_reduction": 1.0 - float(hist[-1]) / float(hist[0]), "batched_domains_per_s": p.D / tb,
        "plain_domains_per_s": sample / tp, "batched_over_plain": (p.D / tb) / (sample / tp),
        "max_rel_V_gap_batched_vs_plain": float(np.max(np.abs(np.array(Vp) - Vb[:sample]) / np.abs(Vb[:sample])))}
    return out


def measure_wide_refinement(local, forward_rate=None):
    """Slope (and split multiplier) refinement on the two wide workloads through the staged reverse
    sweep: per chunk of domains a keep-mode forward pass, then the reverse sweep with its chain
    products on the tensor cores; steps after the first replay one captured step (a context stream of
    its own).  The 16-512x4-8 workload runs at its full horizon (H = 50) on 1024 sub-boxes, from the
    chord slopes (a local minimum of V: V barely moves) and from slopes 0.05 off them; the branch
    workload on 4096 of its domains with split multipliers, batched vs the plain per-domain form.
    `forward_rate`: the bounds pass's domain-steps/s on the same workload, for the ratio."""
    import dataclasses
    from paper_2605_25346_b300 import api

    def run(prob, steps, lrb, start=None, reverse=0):
        r = api.Reach(local, stream=torch.cuda.Stream()).load(prob)
        r.set_options(reverse=reverse)
        if start is not None:
            r.set_alpha(start)
        r.optimize(1, 0.1, lrb)  # warm-up: keep store, scratch and the GEMM tuning
        r.close()
        r = api.Reach(local, stream=torch.cuda.Stream()).load(prob)
        r.set_options(reverse=reverse)
        if start is not None:
            r.set_alpha(start)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = r.optimize(steps, 0.1, lrb)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        res = {"alpha_opt_steps_per_s": steps / t, "domain_steps_per_s": prob.D * prob.H * steps / t,
               "V_first": float(hist[0]), "V_best": float(hist[-1]), "V_reduction": 1.0 - float(hist[-1]) / float(hist[0]),
               "graph_replays": r.graph_replays()}
        return r, res, t

    out = {}
    L16 = wl.large16()
    # the configuration's 10 alpha steps per call; one call also runs a chord-slope pass first and two
    # evaluation passes at the end, so the steady cost of a step is taken from the difference of a
    # 10-step and a 2-step call
    name = "large16 16-512x4-8, 1024 of 262144 sub-boxes, H=50, 10 alpha steps from the chord slopes (staged reverse sweep)"
    prob = dataclasses.replace(L16.subset(np.arange(1024)), H=50)
    r, res, t10 = run(prob, 10, 0.0)  # the chord slopes are a local minimum of V here: V barely moves
    r.close()
    r, _, t2 = run(prob, 2, 0.0)
    r.close()
    per_step = (t10 - t2) / 8.0
    res = {"optimize_call_10_steps_s": t10, "alpha_opt_steps_per_s_whole_call": 10.0 / t10,
           "alpha_step_s": per_step, "alpha_opt_steps_per_s": 1.0 / per_step,
           "domain_steps_per_s": prob.D * prob.H / per_step, "V_first": res["V_first"], "V_best": res["V_best"],
           "V_reduction": res["V_reduction"], "graph_replays": res["graph_replays"],
           "basis": "one step = keep-mode forward pass + staged reverse sweep + projected update, (t(10 steps) - "
                    "t(2 steps)) / 8; a call adds a chord-slope pass and two evaluation passes"}
    if forward_rate:
        res["forward_domain_steps_per_s"] = forward_rate
        res["alpha_step_over_forward"] = res["domain_steps_per_s"] / forward_rate
    out[name] = res
    # the previous engine, the fused reverse kernels out of global slabs, against the staged sweep
    small = dataclasses.replace(L16.subset(np.arange(148)), H=10)
    r, slab, _ = run(small, 2, 0.0, reverse=1)
    r.close()
    r, stg, _ = run(small, 2, 0.0)
    r.close()
    out["large16 16-512x4-8, 148 sub-boxes, H=10: staged vs fused slab reverse"] = {
        "staged_domain_steps_per_s": stg["domain_steps_per_s"], "slab_domain_steps_per_s": slab["domain_steps_per_s"],
        "staged_over_slab": stg["domain_steps_per_s"] / slab["domain_steps_per_s"]}
    # branch domains with split multipliers (alpha + beta), batched vs one domain per call
    name = "branch12 12-256x3-4, 4096 of 65536 branch domains, H=30, alpha+beta (staged reverse sweep)"
    prob = wl.quadrotor_branch(only=np.arange(4096))
    steps, lrb = 2, 0.005
    r, res, t = run(prob, steps, lrb)
    Vb = r.objective()
    r.close()
    sample = 4
    tp, Vp = 0.0, []
    for d in range(sample):
        rr = api.Reach(local).load(prob.subset([d]))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rr.optimize(steps, 0.1, lrb)
        tp += time.perf_counter() - t1
        Vp.append(rr.objective()[0])
        rr.close()
    res.update({"batched_domains_per_s": prob.D / t, "plain_domains_per_s": sample / tp, "plain_sample_domains": sample,
                "batched_over_plain": (prob.D / t) / (sample / tp),
                "max_rel_V_gap_batched_vs_plain": float(np.max(np.abs(np.array(Vp) - Vb[:sample]) / np.abs(Vb[:sample])))})
    out[name] = res
    return out


def measure_tf32_peak(local, n=8192, sustain_s=4.0):
    """Dense TF32 tensor throughput of this GPU: cuBLAS FP32 matmul with TF32 allowed, n^3, best of 10
    (burst) and back to back for `sustain_s` seconds (sustained).  The denominator of the 3xTF32 path."""
    dev = torch.device("cuda", local)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        g = torch.Generator(device=dev).manual_seed(7)
        a = torch.randn(n, n, device=dev, generator=g)
        b = torch.randn(n, n, device=dev, generator=g)
        c = torch.empty(n, n, device=dev)
        for _ in range(3):
            torch.matmul(a, b, out=c)
        torch.cuda.synchronize(dev)
        best = float("inf")
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3)
        reps = max(1, int(sustain_s / best))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        sus = e0.elapsed_time(e1) * 1e-3 / reps
        fl = 2.0 * n ** 3
        return {"tf32_tflops_burst": fl / best / 1e12, "tf32_tflops_sustained": fl / sus / 1e12,
                "how": f"torch.matmul FP32 with TF32 allowed (cuBLAS), {n}^3, best of 10 and {reps} back to back"}
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def measure_wide(local, reps=2, tf32=None):
    """Throughput of the staged tcgen05 path on domain samples of the two wide workloads."""
    from paper_2605_25346_b300 import api
    out = {}
    bf16_burst, bf16_sus, _hbm, basis = peaks()
    peak_tf32 = bf16_burst * 1.1 / 2.25  # nominal TF32/BF16 ratio (1.1 / 2.25 PFLOP/s)
    peak_tf32_sus = bf16_sus * 1.1 / 2.25
    if tf32 is None:
        tf32 = measure_tf32_peak(local)
        out["tf32_peak_measured"] = tf32
    for name, prob in (("branch12 12-256x3-4, 4096 of 65536 branch domains, H=30",
                        wl.quadrotor_branch(only=np.arange(4096))),
                       ("large16 16-512x4-8, 2048 of 262144 sub-boxes, H=50", wl.large16().subset(np.arange(2048)))):
        r = api.Reach(local).load(prob)
        for _ in range(2):  # the plain first call, then the call that captures the CUDA graph
            r.bounds(on_device=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):  # graph replays, as in the headline step
            r.bounds(on_device=True)
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) / reps
        fl = fused_flops_per_domain_step(prob.widths) * prob.D * prob.H
        out[name] = {"domain_steps_per_s": prob.D * prob.H / t, "ms_per_pass": 1e3 * t,
                     "fp32eq_tflops_whole_pass": fl / t / 1e12,
                     "fp32eq_peak_tflops_burst": peak_tf32 / 3.0,
                     "fp32eq_peak_tflops_sustained": peak_tf32_sus / 3.0,
                     "frac_of_fp32eq_tensor_peak_burst": fl / t / 1e12 / (peak_tf32 / 3.0),
                     "frac_of_fp32eq_tensor_peak_sustained": fl / t / 1e12 / (peak_tf32_sus / 3.0),
                     "frac_of_measured_tf32_over_3_burst": fl / t / 1e12 / (tf32["tf32_tflops_burst"] / 3.0),
                     "frac_of_measured_tf32_over_3_sustained": fl / t / 1e12 / (tf32["tf32_tflops_sustained"] / 3.0),
                     "peak_basis": f"3xTF32: one FP32-equivalent FLOP = 3 TF32 tensor FLOPs; TF32 peak = bf16 "
                                   f"{basis} x 1.1/2.25 (nominal ratio); a pass of H={prob.H} steps is a "
                                   f"long, power-capped run, so the sustained figure is the relevant one"}
        r.close()
        # the FP64 oracle on the host cores, on the first domains of the same sample (bounded time)
        cpu = oracle_baseline(prob, target_s=5.0, max_domains=4 if prob.widths[1] >= 512 else 32)
        out[name]["cpu_baseline"] = cpu
        out[name]["gpu_over_cpu"] = out[name]["domain_steps_per_s"] / cpu["value"]
    return out


def full_large16():
    """One pass of the staged tensor-core path over all 262,144 sub-boxes of the 16-512x4-8 workload
    with H = 50 (about 1.1e16 FP32-equivalent FLOP), after one warm-up pass on 2048 of them."""
    from paper_2605_25346_b300 import api
    prob = wl.large16()
    warm = api.Reach(0).load(prob.subset(np.arange(2048)))
    warm.bounds(on_device=True)
    warm.close()
    r = api.Reach(0).load(prob)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = r.bounds(on_device=True)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    fl = fused_flops_per_domain_step(prob.widths) * prob.D * prob.H
    finite = bool(torch.isfinite(out["lo"]).all() and torch.isfinite(out["hi"]).all())
    print(json.dumps({"full_large16": {"domains": prob.D, "horizon": prob.H, "seconds": t,
                                       "domain_steps_per_s": prob.D * prob.H / t, "fp32eq_tflops": fl / t / 1e12,
                                       "all_finite": finite, "launches": r.launches()}}), flush=True)
    r.close()


def wide_refine(domains, horizon):
    """One projected-gradient slope step (keep-mode forward pass and staged reverse sweep, update) on
    the first `domains` sub-boxes of the 16-512x4-8 workload with horizon `horizon` (a profiling case:
    the GEMM launch shapes are the heuristic's, so no tuning trials appear in a launch list)."""
    import dataclasses
    from paper_2605_25346_b300 import api
    prob = dataclasses.replace(wl.large16().subset(np.arange(domains)), H=horizon)
    r = api.Reach(0).load(prob)
    r.set_options(tuning=1)
    t0 = time.perf_counter()
    hist = r.optimize(1, 0.1, 0.0)
    torch.cuda.synchronize()
    print(json.dumps({"wide_refine": {"domains": domains, "horizon": horizon, "seconds": time.perf_counter() - t0,
                                      "V": [float(v) for v in hist], "launches": r.launches()}}), flush=True)
    r.close()


def wide_pass(domains, horizon, gemm_shape=0):
    """Two bounds passes of the staged path on the first `domains` sub-boxes of the 16-512x4-8
    workload with horizon `horizon` (a small case for kernel profiling); `gemm_shape` > 0 forces the
    tensor-core GEMM's launch shape (dr_options.tuning = 100 + shape)."""
    import dataclasses
    from paper_2605_25346_b300 import api
    prob = dataclasses.replace(wl.large16().subset(np.arange(domains)), H=horizon)
    r = api.Reach(0).load(prob)
    if gemm_shape:
        r.set_options(tuning=100 + gemm_shape)
    for _ in range(2):
        r.bounds(on_device=True)
    torch.cuda.synchronize()
    print(json.dumps({"wide_pass": {"domains": domains, "horizon": horizon, "launches": r.launches()}}), flush=True)
    r.close()


def workload(rank=0):
    """The rank's chunk of 16,384 consecutive sub-boxes of the large workload (weak scaling: every
    rank bounds its own chunk; chunks wrap around after the 16 chunks of the grid)."""
    p = wl.large16()
    c0 = (rank * HEADLINE_CHUNK) % p.D
    return p.subset(np.arange(c0, c0 + HEADLINE_CHUNK))


def peaks():
    """(bf16 burst, bf16 sustained, hbm GB/s, basis) from the measured peaks file, else the fallback."""
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(mp["bf16_tflops"]), float(mp["bf16_tflops_sustained"]), float(mp.get("hbm_gbs", 6400.0)), "of measured"
    except Exception:
        return 1800.0, 1400.0, 6400.0, "of fallback"


def measure_quad6(local, steps=10, warmup=3):
    """The 4096-sub-box workload (6-64-64-3, H = 10) on the grouped fused kernel: one launch per
    pass plus the hull, replayed from a CUDA graph; roofline of the fused kernel against FP32 issue."""
    from paper_2605_25346_b300 import api
    prob = wl.quad6_batched()
    D, H, n = prob.D, prob.H, prob.n
    stream = torch.cuda.Stream()
    r = api.Reach(local, stream=stream).load(prob)
    dev = f"cuda:{local}"
    lo = torch.empty(D, H + 1, n, dtype=torch.float64, device=dev)
    hi = torch.empty_like(lo)
    hl = torch.empty(H + 1, n, dtype=torch.float64, device=dev)
    hh = torch.empty_like(hl)
    st = torch.empty(D, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    P = api._ptr

    def step(hull=True):
        r._c(r.lib.dr_compute_bounds(r.ctx, P(lo), P(hi), P(hl) if hull else None, P(hh) if hull else None, P(st), 1))

    out = {}
    with torch.cuda.stream(stream):
        for hull in (True, False):
            for _ in range(warmup):
                step(hull)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for i in range(steps):
                flush.zero_()
                ev[i][0].record(stream)
                step(hull)
                ev[i][1].record(stream)
            torch.cuda.synchronize()
            out[hull] = statistics.mean(a.elapsed_time(b) for a, b in ev)
    r.close()
    flops = fused_flops_per_domain_step(prob.widths) * D * H
    peak = SMS * FP32_LANES_PER_SM * 2 * 2032.0 * 1e6 / 1e12
    achieved = flops / (out[False] * 1e-3) / 1e12
    return {"workload": "quad6 6-64-64-3, 4^6 = 4096 sub-boxes, H=10, chord slopes (grouped fused kernel)",
            "domain_steps_per_s": D * H / (out[True] * 1e-3), "ms_per_step": out[True],
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": FUSED_TRAFFIC_BYTES, "kernel": "k_fused_forward_multi", "kernel_ms": out[False],
                         "peak_basis": "148 SMs x 128 FP32 lanes x 2 FLOP x 2032 MHz (FMA issue rate at max SM clock)"}}


def measure_quad6_fresh(local):
    """measure_quad6 in a fresh process: the short fused launches measured 10-40 % slower inside this
    process after the large staged workload and the TF32 probe had run (same kernel variant, same
    stream setup), and 1.04-1.07 ms per pass in a process of their own."""
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--quad6"], capture_output=True, text=True,
                             timeout=600, env=dict(os.environ, LOCAL_RANK=str(local)))
        for ln in out.stdout.splitlines()[::-1]:
            if ln.startswith("{"):
                res = json.loads(ln)["quad6"]
                res["process"] = "fresh"
                return res
    except (OSError, subprocess.SubprocessError, ValueError, KeyError):
        pass
    res = measure_quad6(local)
    res["process"] = "benchmark process (the fresh-process run failed)"
    return res


def measure_tpush(local, reps=5):
    """DT neural dynamics with planned inputs (the T-pushing-shaped 7-96x3-5 residual model, H = 10):
    bounds over 128 initial boxes and over 1024 MPC action samples, and the gradient dV/du of every
    sample (forward pass with tape plus reverse sweep), batched vs one sample per call."""
    from paper_2605_25346_b300 import api
    out = {}
    for name, prob in (("tpush_dt 128 boxes x action sequences", wl.tpush_dt()),
                       ("tpush_mpc 1024 action samples", wl.tpush_mpc())):
        t, _, _ = _time_passes(local, prob, reps)
        out[name] = {"domain_steps_per_s": prob.D * prob.H / t, "ms_per_pass": 1e3 * t}
    prob = wl.tpush_mpc()
    r = api.Reach(local).load(prob)
    r.backward()  # warm-up: tape and gradient buffers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        r.backward()
        g = r.shift_gradient()
    tb = (time.perf_counter() - t0) / reps
    r.close()
    n = prob.meta["state_dims"]
    sample = 8
    tp = 0.0
    for d in range(sample):
        rr = api.Reach(local).load(prob.subset([d]))
        rr.backward()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rr.backward()
        gp = rr.shift_gradient()
        tp += time.perf_counter() - t1
        # the same gradient (the staged sweep's GEMM launch shapes differ with the batch, which moves
        # FP32 rounding by ~1e-7; the parity tolerance of gradients is 1e-4 of the largest entry)
        assert np.abs(gp[0] - g[d]).max() <= 1e-4 * np.abs(g[d]).max()
        rr.close()
    out["tpush_mpc dV/du"] = {"samples_per_s_batched": prob.D / tb, "ms_per_gradient_batched": 1e3 * tb,
                              "samples_per_s_plain": sample / tp, "plain_sample": sample,
                              "batched_over_plain": (prob.D / tb) / (sample / tp),
                              "max_abs_dV_du": float(np.abs(g[:, :prob.H, n:]).max())}
    return out


def measure_rigorous(local):
    """Rigorous rounding mode (worst-case error bounds carried through the pass): how far its boxes
    lie outside the FP64 oracle's (relative to max(|lo|, |hi|, width) of the oracle's box, the
    default mode's 1e-5 parity scale) and its throughput next to the default mode."""
    import dataclasses
    from oracle import reach as orc
    from paper_2605_25346_b300 import api
    out = {}
    for name, prob, sample in (("quad6 6-64-64-3, 4096 sub-boxes, H=10", wl.quad6_batched(), np.arange(0, 4096, 64)),
                               ("cartpole 4-128-128-2, 1024 sub-boxes, H=20", wl.cartpole_diff(), np.arange(0, 1024, 16)),
                               ("large16 16-512x4-8, 296 sub-boxes, H=50", dataclasses.replace(wl.large16().subset(
                                   np.arange(0, 262144, 886)[:296]), H=50), np.arange(0, 296, 74))):
        res = {}
        for rig in (0, 1):
            stream = torch.cuda.Stream()
            r = api.Reach(local, stream=stream).load(prob)
            r.set_options(mode=prob.mode, rigorous=rig)
            with torch.cuda.stream(stream):
                r.bounds(on_device=True)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                g = r.bounds(on_device=False)
                t = time.perf_counter() - t0
            r.close()
            o = orc.reach(prob.subset(sample))
            olo, ohi = o["lo"].numpy(), o["hi"].numpy()
            scale = np.maximum(np.maximum(np.abs(olo), np.abs(ohi)), ohi - olo)
            dev = np.maximum(olo - g["lo"][sample], g["hi"][sample] - ohi) / scale
            res["rigorous" if rig else "default"] = {
                "domain_steps_per_s": prob.D * prob.H / t, "max_outward_dev_rel": float(dev.max()),
                "median_outward_dev_rel": float(np.median(dev)), "encloses_oracle": bool((dev >= 0).all()),
                "sampled_domains": int(len(sample))}
        out[name] = res
    return out


def _time_passes(local, prob, reps):
    """Seconds per dr_compute_bounds pass (CUDA events; graph replays after two warm calls), the
    last output and the replay count."""
    from paper_2605_25346_b300 import api
    stream = torch.cuda.Stream()
    r = api.Reach(local, stream=stream).load(prob)
    with torch.cuda.stream(stream):
        for _ in range(2):  # the plain first call, then the call that captures the CUDA graph
            r.bounds(on_device=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            out = r.bounds(on_device=True)
        e1.record(stream)
        torch.cuda.synchronize()
    replays = r.graph_replays()
    r.close()
    return e0.elapsed_time(e1) * 1e-3 / reps, out, replays


def measure_branch12_full(local, reps=3):
    """All 65,536 branch domains (0..32 ReLU splits each) of the 12-256x3-4 workload, H = 30, on the
    staged tensor-core path: one dr_compute_bounds per pass, replayed from a CUDA graph.  The same
    domains without their splits, timed the same way, show what the ragged split lists cost."""
    bf_b, bf_s, _, basis = peaks()
    t0 = time.perf_counter()
    prob = wl.quadrotor_branch()
    gen_s = time.perf_counter() - t0
    t, out, replays = _time_passes(local, prob, reps)
    t_nosplit, _, _ = _time_passes(local, wl.quadrotor_branch(with_splits=False), reps)
    counts = np.diff(prob.splits.row_ptr)
    fl = fused_flops_per_domain_step(prob.widths) * prob.D * prob.H
    fp32eq_sus = bf_s * 1.1 / 2.25 / 3.0
    res = {"workload": "branch12 12-256x3-4, all 65,536 branch domains with 0..32 splits (uniform count), H=30",
           "splits_total": int(prob.splits.nnz), "splits_min": int(counts.min()), "splits_max": int(counts.max()),
           "domain_steps_per_s": prob.D * prob.H / t, "ms_per_pass": 1e3 * t, "fp32eq_tflops_whole_pass": fl / t / 1e12,
           "frac_of_fp32eq_tensor_peak_sustained": fl / t / 1e12 / fp32eq_sus,
           "peak_basis": f"bf16 sustained {basis} x 1.1/2.25 / 3", "split_generation_s_host": gen_s,
           "infeasible_domains": int(((out["status"] & 2) != 0).sum().item()),
           "cuda_graph_replays": int(replays),
           "ms_per_pass_same_domains_without_splits": 1e3 * t_nosplit,
           "split_overhead": t / t_nosplit - 1.0}
    return res


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []  # (host time, csv line)
        self.window = (0.0, float("inf"))

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.time() + 5.0  # nvidia-smi needs a moment before its first sample
            while not self.lines and time.time() < t_end:
                time.sleep(0.05)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, start, end):
        """Restrict the summary to samples taken in [start, end] (host time)."""
        self.window = (start, end)

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = [ln for ts, ln in self.lines if self.window[0] - 0.15 <= ts <= self.window[1] + 0.15]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons), "samples": len(sm)}


def oracle_baseline(prob, target_s=10.0, max_domains=None):
    """Time the FP64 oracle, as it stands, on a bounded sample of the workload's domains."""
    from oracle import reach as orc
    D = prob.D if max_domains is None else min(prob.D, max_domains)
    sub = prob.subset(np.arange(D))
    times = []
    t_end = time.perf_counter() + target_s
    while True:
        t0 = time.perf_counter()
        orc.reach(sub)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() >= t_end or len(times) >= 10:
            break
    t = statistics.mean(times)
    return {"value": D * prob.H / t, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{D} of {prob.D} domains x H={prob.H}, {len(times)} repetitions, mean {t:.3f} s"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores (rank 0 only), each step a bounded sample of
    the headline workload (its first domains, full horizon)."""
    if rank != 0:
        return
    from oracle import reach as orc
    prob = workload()
    sample = 4
    sub = prob.subset(np.arange(sample))
    for _ in range(args.warmup):
        orc.reach(sub)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.reach(sub)
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times)
    val = sample * prob.H / t
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"large16 16-512x4-8, chunk of {HEADLINE_CHUNK} of 262,144 sub-boxes, H=50 "
                                   f"(oracle step: {sample}-domain sample)", "domains": sample, "horizon": prob.H},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": f"{sample} of {prob.D} domains x H={prob.H} per step"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def branch_pass(domains, horizon):
    """Two bounds passes of the staged path on the first `domains` branch domains (with their split
    lists) of the 12-256x3-4 workload with horizon `horizon` (a small case for kernel profiling)."""
    import dataclasses
    from paper_2605_25346_b300 import api
    prob = dataclasses.replace(wl.quadrotor_branch(only=np.arange(domains)), H=horizon)
    r = api.Reach(0).load(prob)
    for _ in range(2):
        r.bounds(on_device=True)
    torch.cuda.synchronize()
    print(json.dumps({"branch_pass": {"domains": domains, "horizon": horizon, "launches": r.launches()}}), flush=True)
    r.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the refinement and other-workload measurements")
    ap.add_argument("--wide-refine", nargs=2, type=int, metavar=("DOMAINS", "H"), default=None,
                    help="profiling aid: one slope-refinement step on a 16-512x4-8 sample and exit")
    ap.add_argument("--full-large16", action="store_true",
                    help="one staged pass over all 262,144 sub-boxes of the 16-512x4-8 workload (H = 50)")
    ap.add_argument("--tf32-probe", action="store_true",
                    help="only the cuBLAS TF32 8192^3 throughput probe (the denominator of the 3xTF32 path)")
    ap.add_argument("--gemm-shape", type=int, default=0, choices=range(0, 7),
                    help="with --wide-pass: force the tensor-core GEMM launch shape (1..6, see dr_gemm_tuning_report)")
    ap.add_argument("--wide-pass", nargs=2, type=int, metavar=("DOMAINS", "H"), default=None,
                    help="profiling aid: run two staged tensor-core passes on a 16-512x4-8 sample and exit")
    ap.add_argument("--quad6", action="store_true",
                    help="only the 6-64-64-3 fused-kernel measurement (one JSON line), in a process of its own")
    ap.add_argument("--branch-pass", nargs=2, type=int, metavar=("DOMAINS", "H"), default=None,
                    help="profiling aid: run two staged tensor-core passes on a 12-256x3-4 branch sample and exit")
    args = ap.parse_args()
    if args.quad6:
        print(json.dumps({"quad6": measure_quad6(int(os.environ.get("LOCAL_RANK", "0")))}), flush=True)
        return
    if args.branch_pass:
        return branch_pass(*args.branch_pass)
    if args.wide_pass:
        return wide_pass(*args.wide_pass, gemm_shape=args.gemm_shape)
    if args.wide_refine:
        return wide_refine(*args.wide_refine)
    if args.full_large16:
        return full_large16()
    if args.tf32_probe:
        print(json.dumps({"tf32_probe": measure_tf32_peak(0, sustain_s=0.0)}), flush=True)
        return
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2605_25346_b300 import _lib, api, shard

    prob = workload(rank)
    D, H, n = prob.D, prob.H, prob.n
    stream = torch.cuda.Stream()
    r = api.Reach(local, stream=stream).load(prob)
    dev = f"cuda:{local}"
    lo = torch.empty(D, H + 1, n, dtype=torch.float64, device=dev)
    hi = torch.empty_like(lo)
    hl = torch.empty(H + 1, n, dtype=torch.float64, device=dev)
    hh = torch.empty_like(hl)
    st = torch.empty(D, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    P = api._ptr

    def step():
        r._c(r.lib.dr_compute_bounds(r.ctx, P(lo), P(hi), P(hl), P(hh), P(st), 1))
        if world > 1:
            # the path's only exchange: the hull over every rank's domains (a9), min/max over ranks
            shard.merge_hull(hl, hh)

    with torch.cuda.stream(stream), ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        l0 = r.launches()
        torch.cuda.synchronize()
        h0 = time.time()
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t_wall = time.perf_counter() - t_wall
        clk.mark(h0, time.time())
        launches = r.launches() - l0
        replays = r.graph_replays()
        step_ms = [a.elapsed_time(b) for a, b in ev]

    ms = statistics.mean(step_ms)
    ms_t = torch.tensor([ms], device=dev)
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms = float(ms_t.item())
    value = world * D * H / (ms * 1e-3)

    # roofline of the dominant kernel: one more pass with every tensor-core GEMM launch bracketed by
    # CUDA events on the stream it is launched on (plain launches, no graph)
    r.set_options(mode=prob.mode, timing=1)
    with torch.cuda.stream(stream):
        flush.zero_()
        step()
        torch.cuda.synchronize()
    kt = {}
    for name, cls in (("all", _lib.DR_KT_GEMM_ALL), ("chain", _lib.DR_KT_GEMM_CHAIN), ("final", _lib.DR_KT_GEMM_FINAL),
                      ("other", _lib.DR_KT_GEMM_OTHER)):
        for size, mr in (("", 0), ("_big", BIG_GEMM_ROWS)):
            nl, tms, fl = r.kernel_timing(cls, mr)
            kt[name + size] = {"launches": nl, "ms": tms, "flop": fl}
    r.set_options(mode=prob.mode, timing=0)

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    def pinned(shape, dtype):
        return torch.empty(shape, dtype=dtype, pin_memory=True)

    hlo = pinned((D, H + 1, n), torch.float64)
    hhi = pinned((D, H + 1, n), torch.float64)
    hhl = pinned((H + 1, n), torch.float64)
    hhh = pinned((H + 1, n), torch.float64)
    hst = pinned((D,), torch.int32)
    lo0 = torch.from_numpy(np.ascontiguousarray(prob.lo, dtype=np.float64)).pin_memory()
    hi0 = torch.from_numpy(np.ascontiguousarray(prob.hi, dtype=np.float64)).pin_memory()

    def e2e_step():
        r._c(r.lib.dr_set_boxes(r.ctx, D, P(lo0), P(hi0), 0))
        r._c(r.lib.dr_compute_bounds(r.ctx, P(hlo), P(hhi), P(hhl), P(hhh), P(hst), 0))

    e2e_steps = min(args.steps, 3)
    e2e_step()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = 2 * D * n * 8
    d2h = 2 * D * (H + 1) * n * 8 + 2 * (H + 1) * n * 8 + 4 * D
    r.close()

    bf_b, bf_s, _hbm, basis = peaks()
    # 3xTF32: one FP32-equivalent FLOP is three TF32 tensor FLOPs; TF32 = bf16 x 1.1/2.25 (nominal ratio).
    # The GEMMs run inside a long, power-capped step, so the sustained figure is the denominator.
    peak_sus = bf_s * 1.1 / 2.25 / 3.0
    peak_burst = bf_b * 1.1 / 2.25 / 3.0
    def rate(k):
        return k["flop"] / (k["ms"] * 1e-3) / 1e12 if k["ms"] > 0 else None

    # the dominant kernel: the final-level persistent GEMM (x W_1 fused in its epilogue), which takes
    # the largest share of the GEMM time; its full-size launches (hidden-layer targets)
    fin = kt["final_big"]
    achieved = rate(fin)
    rows_per_launch = fin["flop"] / max(1, fin["launches"]) / (2.0 * 512 * (512 + 16))
    pass_flops = fused_flops_per_domain_step(prob.widths) * D * H
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak_sus, "unit": "TFLOP/s",
            "frac": (achieved / peak_sus) if achieved else None,
            "traffic": GEMM_TRAFFIC_PER_ROW["final"] * rows_per_launch, "traffic_unit": "B per launch",
            "traffic_basis": "dram read + write of one launch over 65,536 rows (ncu, profiles/k_tc_gemm_pp_large16.md) "
                             "scaled by the launch's rows",
            "kernel": "tc::k_tc_gemm_pp<2> (persistent 3xTF32 GEMM of the last chain level, x W_1 in the epilogue; "
                      "launches of the hidden-layer targets)",
            "kernel_launches_timed": fin["launches"], "kernel_ms_avg": fin["ms"] / max(1, fin["launches"]),
            "algorithmic_flops_per_launch": fin["flop"] / max(1, fin["launches"]),
            "unit_of_work": "one stacked Lambda row: 2 x 512 x 512 (tensor) + 2 x 512 x 16 (x W_1) FP32-equivalent "
                            f"FLOP; a launch processes {rows_per_launch:.0f} rows (a lane chunk's domains x 512)",
            "peak_basis": f"bf16 sustained {basis} ({bf_s} TFLOP/s) x 1.1/2.25 (nominal TF32/BF16) / 3 MMAs per "
                          "FP32-equivalent product",
            "frac_burst_peak": (achieved / peak_burst) if achieved else None,
            "timing": "CUDA events around every GEMM launch on its own lane stream, one pass of the same step "
                      "(plain launches); the two lanes run concurrently, so a launch's duration includes the "
                      "other lane's kernels sharing the GPU",
            "chain_level_gemm_big": {"tflops": rate(kt["chain_big"]), "frac": (rate(kt["chain_big"]) or 0) / peak_sus,
                                     "traffic_per_launch": GEMM_TRAFFIC_PER_ROW["chain"] * kt["chain_big"]["flop"] /
                                     max(1, kt["chain_big"]["launches"]) / (2.0 * 512 * 512)},
            "gemm_classes": kt,
            "gemm_share_of_gemm_time": {k: kt[k]["ms"] / max(1e-9, kt["all"]["ms"]) for k in ("chain", "final", "other")},
            "pass_fp32eq_tflops": pass_flops / (ms * 1e-3) / 1e12,
            "pass_frac_of_peak": pass_flops / (ms * 1e-3) / 1e12 / peak_sus}

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = oracle_baseline(prob, target_s=12.0, max_domains=8)
        extras = {}
        if not args.no_extras and world == 1:
            tf32 = measure_tf32_peak(local)
            extras["tf32_peak_measured"] = tf32
            if achieved:
                roof["frac_of_measured_tf32_over_3_sustained"] = achieved / (tf32["tf32_tflops_sustained"] / 3.0)
                roof["frac_of_measured_tf32_over_3_burst"] = achieved / (tf32["tf32_tflops_burst"] / 3.0)
                roof["frac_named"] = ("frac uses the bf16-derived sustained peak; frac_of_measured_tf32_over_3_* use "
                                      "the cuBLAS TF32 probe of this run")
            roof["pass_frac_of_measured_tf32_over_3_sustained"] = roof["pass_fp32eq_tflops"] / (tf32["tf32_tflops_sustained"] / 3.0)
            extras["quad6"] = measure_quad6_fresh(local)
            extras["branch12_full"] = measure_branch12_full(local)
            extras["tpush_dt_mpc"] = measure_tpush(local)
            extras["rigorous"] = measure_rigorous(local)
            extras["refinement"] = measure_refinement(local)
            extras["wide"] = measure_wide(local, tf32=tf32)
            extras["wide_refinement"] = measure_wide_refinement(local, forward_rate=value / world)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32(3xtf32)+f64", "data": "synthetic",
                "config": {"workload": f"large16 16-512x4-8, chunk of {D} of 262,144 sub-boxes per GPU, H={H}, "
                                       "chord slopes", "domains_per_gpu": D, "horizon": H,
                           "l2": "flushed between timed steps (working set 16 GiB, also above L2)",
                           "parallelism": f"domains sharded over {world} rank(s); per step one min/max all-reduce of "
                                          "the (H+1) x n hull when N > 1"},
                "e2e": {"value": world * D * H / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "steps": e2e_steps},
                "gpu_launches": int(launches),
                "cuda_graph_replays": int(replays),
                "gemm_autotuner_picks": api.gemm_tuning_report().strip().split("\n"),
                "wall_ms_per_step_incl_flush": 1e3 * t_wall / args.steps,
                "roofline": roof, "cpu_baseline": cpu, "clocks": clk.summary(), "extras": extras}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
