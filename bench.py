#!/usr/bin/env python
"""Throughput of the nested Krylov-Ritz sign function sgn(gamma5 D_w(mu)) b on GB300.

One step = one batched solve of the workload's n_rhs sources (12 spin-colour
point sources at the origin) by the nested method: outer two-sided Lanczos
(two-float stencil for the first j0 steps, FP32 stencil after; the
recurrence itself two-float from step j1 on, FP64 before), one p for the
batch, LU of p H_k, inner two-sided Lanczos with H_k', batched
Roberts-Higham (FP64), two-float lift.  The whole solve replays one CUDA
graph; --inflight batches (default 4) run at a time on their own streams.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                    [--inflight B] [--j1 J] [--tune-cache FILE] [--mode bench|ncu]

Prints one JSON line on rank 0.  Under torchrun each rank runs an independent
replica of the workload on its own GPU (the method has no exchange step:
"replicas only"); the timing is the max over ranks.
"""
from __future__ import annotations

import os

# The CPU oracle leg uses one host thread (numpy elementwise code is single
# threaded; this keeps its BLAS calls single threaded too).
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sgn(A)b solves/s at rel err ≤1e-8, mixed+batched vs FP64 plain; stencil %HBM"
TOL = 1e-8
REF_BUDGET_S = 120.0

WORKLOADS = {
    # 8^4, mu = 0.3 (two-sided), 12 point sources, mixed precision, one graph
    # k and the FP32 switch j0 are the smallest (from a sweep) that give rel err
    # <= 1e-8 on all 12 sources with these links; the whole recurrence runs in
    # two-float arithmetic (j1 = 0: the same errors as j1 = j0 here)
    "8^4-mu0.3-12pt": dict(dims=(8, 8, 8, 8), mu=0.3, m_w=-2.0, link_seed=103, k=896, ell=160, j0=256, j1=0,
                           n_rhs=12, source="point", mixed=True),
    "8^4-mu0-12pt": dict(dims=(8, 8, 8, 8), mu=0.0, m_w=-2.0, link_seed=103, k=768, ell=160, j0=64,
                         n_rhs=12, source="point", mixed=True),
}
DEFAULT_WORKLOAD = "8^4-mu0.3-12pt"
# stencil roofline case: 16^3 x 32, FP32 stencil, 12 RHS in one launch (A and A^dagger)
STENCIL_DIMS = (16, 16, 16, 32)


def max_over_ranks(ms, dist=None):
    """The timed region's length: the maximum over the ranks (replicas: each rank
    solves its own batch; this reduction and the barriers are the only
    collectives)."""
    if not dist:
        return ms
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(solves_per_step, steps, ms, world):
    """Solves/s of the whole job: every rank solves solves_per_step sources per
    step (weak scaling), over the slowest rank's time."""
    return world * solves_per_step * steps / (ms * 1e-3)


def profiled_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summaries
    (a line 'traffic_bytes_per_launch <kernel>: <bytes>'), else None."""
    import glob
    import re
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                m = re.match(r"\s*traffic_bytes_per_launch\s+(\S+):\s*([0-9.eE+]+)", line)
                if m and m.group(1) == kernel:
                    return float(m.group(2))
    return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(w):
    import inputs
    U, eps = inputs.su3_links(w["dims"], w["link_seed"])
    if w["source"] == "point":
        b = inputs.point_sources(w["dims"])[: w["n_rhs"]]
    else:
        b = inputs.gaussian_sources(w["dims"], w["link_seed"] + 100, n_rhs=w["n_rhs"])
    return U, b


def oracle_leg(w, U, b, budget_s=40.0):
    """The CPU oracle, as it stands, on a bounded sample: the nested method for
    the first source of the workload (same k, l), one host thread."""
    from oracle import nested
    t0 = time.perf_counter()
    y, info = nested.sign_apply(U, w["dims"], w["mu"], w["m_w"], b[0], w["k"], w["ell"])
    t = time.perf_counter() - t0
    return y, t


def run_reference(args, w, rank):
    """The oracle as it stands, on the host cores, as the reference arm.

    A full oracle solve of one source takes tens of seconds, so each step is
    a bounded sample of the workload: the oracle's outer recurrence (App. B,
    two-sided for mu != 0), which is the bulk of its time and linear in k,
    for k_s of the k steps, from source (step mod n_rhs); the metric counts
    k_s / k of a solve per step.  k_s is sized from a short calibration so
    that warm-up plus timed steps take about REF_BUDGET_S seconds.  The
    inner part (p estimate, LU, inner Lanczos, RHi: a few percent of the
    oracle's time) is left out of the sample, which favours the reference."""
    if rank != 0:
        return 0
    from oracle import nested
    U, b = make_inputs(w)
    apply_a, apply_adag, herm = nested.operator(U, w["dims"], w["mu"], w["m_w"])
    t0 = time.perf_counter()
    nested.outer_basis(apply_a, apply_adag, b[0], 8, herm)
    per_step = (time.perf_counter() - t0) / 8
    steps, warm = max(1, args.steps), max(0, args.warmup)
    k_s = int(np.clip(REF_BUDGET_S / (steps + warm) / per_step, 8, w["k"]))
    times = []
    for i in range(warm + steps):
        t0 = time.perf_counter()
        nested.outer_basis(apply_a, apply_adag, b[i % len(b)], k_s, herm)
        if i >= warm:
            times.append(time.perf_counter() - t0)
    tot = float(np.sum(times))
    value = steps * (k_s / w["k"]) / tot
    sample = ("oracle outer recurrence (numpy FP64, one thread), %d of the k = %d steps per step, one source "
              "per step; the metric counts %d/%d of a solve per step" % (k_s, w["k"], k_s, w["k"]))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * tot / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w, args),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def j1_of(w, args):
    """First outer step whose recurrence runs in two-float arithmetic."""
    j1 = args.j1 if args.j1 is not None else w.get("j1", -1)
    return w["j0"] if j1 < 0 else min(j1, w["j0"])


def config_of(w, args):
    return {"workload": args.workload, "lattice": "x".join(str(d) for d in w["dims"]), "mu": w["mu"],
            "m_w": w["m_w"], "k": w["k"], "ell": w["ell"], "n_rhs": w["n_rhs"],
            "sources": "12 spin-colour point sources at the origin" if w["source"] == "point" else "gaussian",
            "links": "U = exp(i eps X), plaquette 0.59, seed %d" % w["link_seed"],
            "precision": ("two-float (48-bit) stencil for outer steps < %d, FP32 stencil after; the recurrence "
                          "(vector updates, inner products, basis) FP64 before step %d and two-float from it on; "
                          "H_k, p, LU of pH_k, inner Lanczos and RHi FP64; lift two-float"
                          % (w["j0"], j1_of(w, args))) if w["mixed"] else "FP64",
            "p": "one p per batch: Eq. popt with z_min, z_max of A estimated as the extremes over the "
                 "batch's H_k (power / inverse iteration)",
            "graph": True, "parallelism": "replicas" if args.gpus > 1 else "single",
            "batches_in_flight": args.inflight,
            "l2": "working set (Krylov basis %.1f GB) larger than L2" % (
                12 * w["n_rhs"] * np.prod(w["dims"]) * w["k"] * 16 / 1e9)}


def stencil_roofline(nk, torch, peaks):
    """The solver's stencil kernel (FP32 Wilson stencil for 12 RHS of A and 12
    of A^dagger in one launch, fused with the first half of the Lanczos step)
    on 16^3 x 32, a lattice whose vectors are larger than L2.  Achieved
    algorithmic GB/s from CUDA events around each launch on the launch stream
    (NK_PROFILE), over a 16-step mixed solve with every stencil in FP32.

    Algorithmic bytes of launch j (each array moved once): FP32 links 288 B/site;
    per right vector FP32 input 96, FP64 q_{j-1} 192 (j > 0), FP64 dot vector
    p_j 192, FP64 output r 192 (j < k-1); per left vector (j < k-1) FP32 input
    96, FP64 p_{j-1} 192 (j > 0), FP64 output 192."""
    import inputs
    dims = STENCIL_DIMS
    ctx = nk.Context(dims)
    ctx.load_links(inputs.su3_links(dims, 105)[0])
    ctx.set_mu_mw(0.2, -2.0)
    V = int(np.prod(dims))
    n = 12
    ctx.autotune(n, nk.NK_MIXED)
    b = torch.zeros((n, 12 * V), dtype=torch.complex128, device="cuda")
    b[:, :12] = torch.eye(12, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(b)
    k = 16
    ctx.set_precision(0)
    ctx.sign_apply_dev(b, y, n, k, 4, flags=nk.NK_MIXED | nk.NK_PROFILE)
    st, _ = ctx.sign_apply_dev(b, y, n, k, 4, flags=nk.NK_MIXED | nk.NK_PROFILE)
    torch.cuda.synchronize()
    t_ms = st["t_class_ms"]["dslash"]
    launches = st["n_class"]["dslash"]
    total = 0
    for j in range(k):
        bj = 288 + n * (96 + (192 if j > 0 else 0) + 192 + (192 if j < k - 1 else 0))
        if j < k - 1:
            bj += n * (96 + (192 if j > 0 else 0) + 192)
        total += V * bj
    gbs = total / (t_ms * 1e-3) / 1e9
    ctx.close()
    return {"kernel": "k_dslash_step1<float, two-sided> (12 RHS A + 12 RHS A^dagger per launch)",
            "lattice": "16x16x16x32", "bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs"),
            "unit": "GB/s", "frac": gbs / peaks.get("hbm_gbs", 6800.0), "ms_per_launch": t_ms / launches,
            "bytes_per_launch": total / launches, "launches": launches}


def run_gpu(args, w, rank, world, local_rank):
    import torch
    import paper_0912_4457_gb300 as nk
    from paper_0912_4457_gb300 import build as nkbuild
    if not os.path.exists(nkbuild.LIB) or not nkbuild.up_to_date():
        if rank == 0:
            nkbuild.build()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    peaks = measured_peaks()
    U, b_host = make_inputs(w)
    n_rhs, k, ell = w["n_rhs"], w["k"], w["ell"]
    flags = (nk.NK_MIXED if w["mixed"] else nk.NK_FP64) | nk.NK_SHARED_P
    ctx = nk.Context(w["dims"])
    ctx.load_links(U)
    ctx.set_mu_mw(w["mu"], w["m_w"])
    ctx.set_precision(w.get("j0", -1))
    ctx.set_df_recurrence(j1_of(w, args))
    # launch shape of the outer recurrence: timed on 16 synthetic steps, kept
    shape, tune_ms = ctx.autotune(n_rhs, flags, args.tune_cache)
    stream = torch.cuda.current_stream()
    b_dev = torch.from_numpy(np.ascontiguousarray(b_host)).cuda()
    y_dev = torch.zeros_like(b_dev)
    # Batches in flight: each step is one whole batched solve; with two contexts
    # on two streams the next batch's outer recurrence (all SMs) runs while the
    # previous batch's inner part and RHi (12 and 96 SMs) finish.
    inflight = max(1, args.inflight)
    ctxs, ys, streams = [ctx], [y_dev], [torch.cuda.Stream() for _ in range(inflight)]
    for _ in range(1, inflight):
        c2 = nk.Context(w["dims"])
        c2.load_links(U)
        c2.set_mu_mw(w["mu"], w["m_w"])
        c2.set_precision(w.get("j0", -1))
        c2.set_df_recurrence(j1_of(w, args))
        c2.set_launch(n_rhs, flags, *shape)
        ctxs.append(c2)
        ys.append(torch.zeros_like(b_dev))
    for _ in range(args.warmup):
        for c_, y_ in zip(ctxs, ys):
            st, _ = c_.sign_apply_dev(b_dev, y_, n_rhs, k, ell, flags=flags)
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s_ in streams:
        s_.wait_stream(stream)
    launches = 0
    for i in range(args.steps):
        c_ = ctxs[i % inflight]
        if inflight > 1:
            if i >= inflight:       # the previous batch of this context
                st, _ = c_.wait()
                launches += st["launches"]
            c_.sign_apply_dev(b_dev, ys[i % inflight], n_rhs, k, ell, flags=flags | nk.NK_ASYNC,
                              stream=streams[i % inflight])
        else:
            st, _ = c_.sign_apply_dev(b_dev, y_dev, n_rhs, k, ell, flags=flags)
            launches += st["launches"]
    if inflight > 1:
        for c_ in ctxs:
            st, rc_w = c_.wait()
            launches += st["launches"]
        for s_ in streams:
            stream.wait_stream(s_)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    y = y_dev.cpu().numpy()
    for c_ in ctxs[1:]:
        c_.close()
    # latency of one batch with nothing else in flight
    l0 = torch.cuda.Event(enable_timing=True)
    l1 = torch.cuda.Event(enable_timing=True)
    l0.record(stream)
    for _ in range(2):
        ctx.sign_apply_dev(b_dev, y_dev, n_rhs, k, ell, flags=flags)
    l1.record(stream)
    torch.cuda.synchronize()
    latency_ms = l0.elapsed_time(l1) / 2

    # e2e: host buffers in pinned memory, through the host-pointer C entry point
    b_pin = torch.from_numpy(np.ascontiguousarray(b_host)).pin_memory()
    y_pin = torch.zeros_like(b_pin).pin_memory()
    bp, yp = b_pin.numpy(), y_pin.numpy()
    ctx.sign_apply(bp, k, ell, flags=flags)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        _lib_host_solve(ctx, bp, yp, k, ell, flags)
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    # comparator named by the metric: the plain all-FP64 nested method, one
    # source per solve, same k and l, on the same GPU (source 0)
    b1 = b_dev[:1].contiguous()
    y1 = torch.zeros_like(b1)
    ctx.sign_apply_dev(b1, y1, 1, k, ell, flags=nk.NK_FP64)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    nrep = 2
    f0.record(stream)
    for _ in range(nrep):
        ctx.sign_apply_dev(b1, y1, 1, k, ell, flags=nk.NK_FP64)
    f1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = f0.elapsed_time(f1) / nrep
    y_fp64 = y1.cpu().numpy()[0]

    # per-kernel-class device times (NK_PROFILE: CUDA events around each launch)
    stp, _ = ctx.sign_apply_dev(b_dev, y_dev, n_rhs, k, ell, flags=flags | nk.NK_PROFILE)
    torch.cuda.synchronize()
    if rank != 0:
        ctx.close()
        return 0

    # accuracy: the oracle on source 0 (this is also the timed CPU baseline sample)
    y_or, t_or = oracle_leg(w, U, b_host)
    err0 = float(np.linalg.norm(y[0] - y_or) / np.linalg.norm(y_or))
    # the paper's sgn^2 estimate (Sec. 3) for all sources: apply the solve to y
    yy = torch.zeros_like(y_dev)
    y_src = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    ctx.sign_apply_dev(y_src, yy, n_rhs, k, ell, flags=flags)
    torch.cuda.synchronize()
    x2 = yy.cpu().numpy()
    eps = [float(np.linalg.norm(x2[i] - b_host[i]) / (2 * np.linalg.norm(b_host[i]))) for i in range(n_rhs)]
    err_fp64 = float(np.linalg.norm(y_fp64 - y_or) / np.linalg.norm(y_or))
    ok = sum(1 for e in eps if e <= TOL)
    if err0 > TOL:
        ok = 0
    solves_per_step = ok

    value = whole_job_value(solves_per_step, args.steps, ms, world)
    e2e_value = solves_per_step / e2e_s
    tc = stp["t_class_ms"]
    nc = stp["n_class"]
    tot = sum(tc.values())
    share = {kk: (tc[kk] / tot if tot else 0.0) for kk in tc}
    dom = max(tc, key=lambda kk: tc[kk])
    roof = dominant_roofline(dom, tc, nc, w, peaks, clocks.get("sm_mhz"))
    sten = stencil_roofline(nk, torch, peaks)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "latency_ms_one_batch": latency_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic", "config": config_of(w, args),
        "accuracy": {"rel_err_vs_oracle_src0": err0, "eps_sgn2_max": max(eps), "solves_meeting_tol": ok,
                     "tol": TOL},
        "e2e": {"value": e2e_value, "unit": "solves/s",
                "h2d_bytes_per_step": int(b_host.nbytes), "d2h_bytes_per_step": int(b_host.nbytes)},
        "fp64_plain": {"value": (1.0 / (fp64_ms * 1e-3)) if err_fp64 <= TOL else 0.0, "unit": "solves/s",
                       "ms_per_solve": fp64_ms, "rel_err_vs_oracle_src0": err_fp64,
                       "what": "same method, all FP64, one source per solve, same k and l, same GPU"},
        "speedup_vs_fp64_plain": (value / world) / (1.0 / (fp64_ms * 1e-3)),
        "gpu_launches": launches,
        "launch_shape": {"stencil_threads": shape[0], "stencil_order": shape[1], "step2_blocks": shape[2],
                         "early_threads": shape[3], "early_order": shape[4], "stencil_split": shape[5],
                         "early_split": shape[6],
                         "autotune_ms_per_outer_step": tune_ms},
        "rhi_iters": stp["rhi_iters"],
        "kernel_class_ms": {kk: round(v, 3) for kk, v in tc.items()},
        "roofline": roof,
        "stencil_roofline": sten,
        "kernel_time_share": {kk: round(v, 4) for kk, v in share.items()},
        "cpu_baseline": {"value": 1.0 / t_or, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": "nested method (numpy FP64 oracle) on source 0 of the workload, same k and l, "
                                   "%.1f s" % t_or},
        "clocks": clocks,
    }
    print(json.dumps(line))
    ctx.close()
    return 0


def run_ncu(args, w):
    """--warmup kernel-by-kernel solves, then one more: the launches an ncu
    launch list or capture selects from (skip the warm-up ones with -s).
    --ncu-k K shortens the outer recurrence to K steps (the per-launch work of
    every kernel but the lift is unchanged; the basis then takes K/k of the
    memory), for captures that must stay small."""
    import torch
    import paper_0912_4457_gb300 as nk
    if args.ncu_k:   # half of the shortened recurrence in each stencil precision
        w = dict(w, k=args.ncu_k, ell=min(w["ell"], args.ncu_k), j0=min(w["j0"], args.ncu_k // 2))
    U, b_host = make_inputs(w)
    ctx = nk.Context(w["dims"])
    ctx.load_links(U)
    ctx.set_mu_mw(w["mu"], w["m_w"])
    ctx.set_precision(w.get("j0", -1))
    ctx.set_df_recurrence(j1_of(w, args))
    flags = (nk.NK_MIXED if w["mixed"] else nk.NK_FP64) | nk.NK_SHARED_P | nk.NK_NO_GRAPH
    # with --tune-cache from a plain bench run the shape is read, not timed
    ctx.autotune(w["n_rhs"], flags, args.tune_cache)
    b_dev = torch.from_numpy(np.ascontiguousarray(b_host)).cuda()
    y_dev = torch.zeros_like(b_dev)
    for _ in range(args.warmup + 1):
        st, _ = ctx.sign_apply_dev(b_dev, y_dev, w["n_rhs"], w["k"], w["ell"], flags=flags)
    torch.cuda.synchronize()
    print("launches per solve %d, device ms %.3f" % (st["launches"], st["t_total_ms"]), file=sys.stderr)
    ctx.close()
    return 0


def _lib_host_solve(ctx, bp, yp, k, ell, flags):
    import ctypes
    from paper_0912_4457_gb300 import nksign
    st = nksign.NkStats()
    rc = ctx._lib.nk_sign_apply(ctx.h, nksign._dptr(bp.view(np.float64)), bp.shape[0], int(k), int(ell), 0.0,
                                0.0, int(flags), nksign._dptr(yp.view(np.float64)), ctypes.byref(st))
    ctx._check(rc)


def dominant_roofline(dom, tc, nc, w, peaks, sm_mhz):
    """Roofline entry for the kernel class with the largest device time.

    Algorithmic work per launch, n_rhs sources, two-sided (Hermitian in
    parentheses); each array moved once, each flop of the method counted once:
      dslash_df: the two-float stencil, 1320 flops per site and vector
             (2 n_rhs (n_rhs) vectors).  Two-float arithmetic costs 11 FP32
             instructions per add and 7 per multiply (TwoSum / FMA-TwoProd
             with renormalisation), 9 on average for the stencil's equal mix, so
             its ALU peak is the FP32 issue rate / 9:
             152 SMs x 128 lanes x f_SM / 9 (f_SM the median SM clock sampled
             during the timed region);
      dslash (FP32 stencil fused with step 1): per site links 288 B + per
             vector FP32 input 96 B, FP64 q_{j-1} and dot vector 2 x 192 B,
             FP64 output 192 B -- HBM;
      step2: 24 (8) FP64 flops per element -- FP64 ALU, 1.0 TFLOP/s measured
             DFMA rate;
      step2_df: reads q_j, r, p_j, l and writes r, l (two-float rings), the
             basis column and, before an FP32 stencil, the FP32 copies: 128
             (64) B per element, 112 (56) without the copies -- HBM;
      lift: reads V_k once, 16 B x k per element -- HBM.
    """
    V = int(np.prod(w["dims"]))
    N = 12 * V
    n_rhs = w["n_rhs"]
    two = w["mu"] != 0.0
    nv = (2 if two else 1) * n_rhs
    ms = tc[dom] / max(1, nc[dom])
    fp64_peak = 1.0  # TFLOP/s, measured DFMA rate of this GB300
    hbm = peaks.get("hbm_gbs", 6800.0)
    if dom == "dslash_df":
        flops = 1320.0 * V * nv
        tf = flops / (ms * 1e-3) / 1e12
        peak = 152 * 128 * (sm_mhz or 2070.0) * 1e6 / 9.0 / 1e12
        return {"kernel": "k_dslash_step1<df> (two-float stencil fused with step 1)", "bound": "alu",
                "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                "traffic": profiled_traffic("k_dslash_step1<df>"),
                "ms_per_launch": ms, "flops_per_launch": flops,
                "peak_derivation": "FP32 issue rate 152 x 128 x f_SM over 9 FP32 instructions per two-float flop"}
    if dom == "step2_df":
        # launches j1 <= j <= k - 2; those with j + 1 >= j0 also write the FP32
        # copy the next (FP32) stencil reads, the others do not
        k, j0 = w["k"], w["j0"]
        j1 = w.get("j1", -1)
        j1 = j0 if j1 < 0 else min(j1, j0)
        n_df = max(1, k - 1 - j1)
        n_copy = min(n_df, k - j0)
        per_el = ((n_copy * (128 if two else 64) + (n_df - n_copy) * (112 if two else 56)) / n_df)
        b = per_el * N * n_rhs
        gbs = b / (ms * 1e-3) / 1e9
        return {"kernel": "k_step2_df (two-float step 2 on the rings)", "bound": "hbm",
                "achieved": gbs, "peak": peaks.get("hbm_gbs"), "unit": "GB/s", "frac": gbs / hbm,
                "traffic": profiled_traffic("k_step2_df"), "ms_per_launch": ms,
                "algorithmic_bytes_per_launch": b}
    if dom == "step2":
        flops = (24 if two else 8) * N * n_rhs
        tf = flops / (ms * 1e-3) / 1e12
        return {"kernel": "k_step2", "bound": "alu", "achieved": tf, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": tf / fp64_peak, "traffic": profiled_traffic("k_step2"), "ms_per_launch": ms,
                "algorithmic_bytes_per_launch": (112 if two else 56) * N * n_rhs}
    if dom in ("dslash", "dslash64"):
        b = V * (288 + nv * (96 + 192)) + V * n_rhs * 2 * 192
        gbs = b / (ms * 1e-3) / 1e9
        return {"kernel": "k_dslash_step1", "bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs"),
                "unit": "GB/s", "frac": gbs / hbm, "traffic": profiled_traffic("k_dslash_step1<float>"),
                "ms_per_launch": ms}
    if dom == "lift":
        b = n_rhs * w["k"] * N * 16
        gbs = b / (ms * 1e-3) / 1e9
        return {"kernel": "k_lift", "bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs"),
                "unit": "GB/s", "frac": gbs / hbm, "traffic": None, "ms_per_launch": ms}
    return {"kernel": dom, "bound": "alu", "achieved": None, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": None, "traffic": None, "ms_per_launch": ms}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--mode", choices=["bench", "ncu"], default="bench",
                    help="ncu: run --warmup solves and then one solve kernel by kernel (no graph, no oracle, "
                         "no output line), for launch lists and captures under ncu")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--ncu-k", type=int, default=0, help="--mode ncu: outer steps (0: the workload's k)")
    ap.add_argument("--j1", type=int, default=None,
                    help="first outer step with a two-float recurrence (default: the workload's)")
    ap.add_argument("--inflight", type=int, default=4,
                    help="batches in flight (contexts on their own streams); 1: one synchronous solve per step")
    ap.add_argument("--tune-cache", default=None,
                    help="launch-shape cache file (read if it has the workload's shape, else written)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    w = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w, rank)
    if args.mode == "ncu":
        return run_ncu(args, w)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    rc = run_gpu(args, w, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
