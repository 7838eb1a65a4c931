#!/usr/bin/env python
"""Throughput of the nested Krylov-Ritz sign function sgn(gamma5 D_w(mu)) b on GB300.

One step = one batched solve of the workload's n_rhs sources (12 spin-colour
point sources at the origin) by the nested method (Eq. nested, App. C steps
2-6): outer two-sided Lanczos (two-float stencil for the first j0 steps,
FP32 stencil after; the recurrence -- vector updates, inner products and
their accumulation, the basis -- in FP64), one p for the batch, LU of p H_k,
inner two-sided Lanczos with H_k', batched Roberts-Higham and the lift, all
FP64.  The whole solve replays one CUDA graph; --inflight batches (default 4)
run at a time on their own streams.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                    [--workload NAME] [--inflight B] [--tune-cache FILE] [--mode bench|ncu]
                    [--quick]

Prints one JSON line on rank 0.  Under torchrun each rank runs an independent
replica of the workload on its own GPU (the method has no exchange step:
"replicas only"); the timing is the max over ranks.
"""
from __future__ import annotations

import os

# numpy in the oracle legs: one BLAS thread per process (the all-cores CPU
# baseline runs one process per core instead)
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
CPU_SAMPLE_S = 12.0
# nominal FP64 rate of GB300 (dense, all SMs): the peak of the FP64-ALU-bound kernels
FP64_PEAK_TFLOPS = 1.25

WORKLOADS = {
    # 10^4, mu = 0.2, 12 point sources: the largest lattice of the paper's
    # range that holds the stored basis (k = 1024: 23.6 GB per batch).  FP64
    # converges by k = 1024 (1e-11 against k = 1536); the FP32 switch j0 sets
    # the error of the mixed schedule (j0 = 128: 2.9e-8, 256: 1.5e-9,
    # 384: 6e-11 against FP64 k = 1536), l = 128 leaves it unchanged.
    # A second nested level l_2 = 64 below l = 128 (Sec. 4.5) leaves the error
    # unchanged (1.55e-9) and halves the size of the RHi matrix.
    "10^4-mu0.2-12pt": dict(dims=(10, 10, 10, 10), mu=0.2, m_w=-2.0, link_seed=104, k=1024, ell=128, nest=(64,),
                            j0=256, j1=-1, n_rhs=12, source="point", mixed=True, k_ref=1536, ell_ref=256),
    # 8^4, mu = 0.3 (two-sided), 12 point sources
    "8^4-mu0.3-12pt": dict(dims=(8, 8, 8, 8), mu=0.3, m_w=-2.0, link_seed=103, k=896, ell=160, j0=256, j1=-1,
                           n_rhs=12, source="point", mixed=True, k_ref=1280, ell_ref=256),
    "8^4-mu0-12pt": dict(dims=(8, 8, 8, 8), mu=0.0, m_w=-2.0, link_seed=103, k=768, ell=160, j0=64, j1=-1,
                         n_rhs=12, source="point", mixed=True, k_ref=1280, ell_ref=256),
}
DEFAULT_WORKLOAD = "10^4-mu0.2-12pt"
# stencil roofline case: 16^3 x 32 (vectors larger than L2), FP32, 12 RHS of A and 12 of A^dagger
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


# ---- oracle legs (CPU; spawned processes, never forked after CUDA is up) ----------

def _oracle_solve(args):
    """The nested oracle on one source (same k, l, nested levels and p as the
    GPU batch)."""
    U, dims, mu, m_w, b0, k, ell, p, ells = args
    from oracle import nested
    t0 = time.perf_counter()
    y, _ = nested.sign_apply(U, dims, mu, m_w, b0, k, ell, p=p, ells=ells)
    return y, time.perf_counter() - t0


def _oracle_steps(args):
    """k_s steps of the oracle's outer recurrence (App. B) from one source: the
    bulk of the oracle's time, linear in k."""
    dims, mu, m_w, link_seed, src, k_s = args
    from oracle import nested
    import inputs
    U, _ = inputs.su3_links(dims, link_seed)
    b = inputs.point_sources(dims)[src]
    a, adag, herm = nested.operator(U, dims, mu, m_w)
    t0 = time.perf_counter()
    nested.outer_basis(a, adag, b, k_s, herm)
    return time.perf_counter() - t0


def cpu_baselines(w, budget_s=CPU_SAMPLE_S):
    """The oracle as it stands on the host cores, on a bounded sample: its outer
    recurrence for k_s of the k steps per source (calibrated to about budget_s
    seconds), (a) one source in one process (1 thread), (b) one source per
    process on every host core.  Each counts k_s / k of a solve per source (the
    inner part, a few percent of the oracle's time, is left out, which favours
    the oracle).  Returns both as solves/s."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    cores = os.cpu_count() or 1
    with ctx.Pool(1) as pool:
        per_step = pool.map(_oracle_steps, [(w["dims"], w["mu"], w["m_w"], w["link_seed"], 0, 8)])[0] / 8
        k_s = int(np.clip(budget_s / per_step, 8, w["k"]))
        t1 = pool.map(_oracle_steps, [(w["dims"], w["mu"], w["m_w"], w["link_seed"], 0, k_s)])[0]
    one = (k_s / w["k"]) / t1
    n_all = cores
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        pool.map(_oracle_steps, [(w["dims"], w["mu"], w["m_w"], w["link_seed"], i % w["n_rhs"], k_s)
                                 for i in range(n_all)])
        tall = time.perf_counter() - t0
    allc = n_all * (k_s / w["k"]) / tall
    sample = ("oracle outer recurrence (numpy FP64), %d of the k = %d steps of a point source per process; "
              "counts %d/%d of a solve per source" % (k_s, w["k"], k_s, w["k"]))
    return ({"value": one, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample + ", 1 process",
             "seconds": t1},
            {"value": allc, "unit": "solves/s", "cores": cores, "kind": "oracle",
             "sample": sample + ", %d processes on %d cores" % (n_all, cores), "seconds": tall})


def run_reference(args, w, rank):
    """The oracle as it stands, on the host cores, as the reference arm.

    A full oracle solve of one 10^4 source takes minutes, so each step is a
    bounded sample of the workload: the oracle's outer recurrence (App. B,
    two-sided for mu != 0), the bulk of its time and linear in k, for k_s of
    the k steps, from source (step mod n_rhs); the metric counts k_s / k of a
    solve per step.  k_s is sized from a short calibration so that warm-up
    plus timed steps take about REF_BUDGET_S seconds.  The inner part (p
    estimate, LU, inner Lanczos, RHi: a few percent of the oracle's time) is
    left out of the sample, which favours the reference."""
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
    """First outer step whose recurrence runs in two-float arithmetic (-1: none,
    the recurrence is FP64 throughout)."""
    j1 = args.j1 if args.j1 is not None else w.get("j1", -1)
    return -1 if j1 < 0 else j1


def precision_text(w, j1):
    if not w["mixed"]:
        return "FP64"
    rec = ("the recurrence (vector updates, inner products and their accumulation, basis V_k) FP64"
           if j1 < 0 else
           "the recurrence FP64 before step %d and two-float (about 48-bit) from it on, lift two-float" % j1)
    return ("two-float (about 48-bit) stencil for outer steps < %d, FP32 stencil after; %s; H_k, p, LU of "
            "pH_k, inner Lanczos, RHi%s FP64" % (w["j0"], rec, " and lift" if j1 < 0 else ""))


def config_of(w, args):
    return {"workload": args.workload, "lattice": "x".join(str(d) for d in w["dims"]), "mu": w["mu"],
            "m_w": w["m_w"], "k": w["k"], "ell": w["ell"], "j0": w["j0"], "n_rhs": w["n_rhs"],
            "sources": "12 spin-colour point sources at the origin" if w["source"] == "point" else "gaussian",
            "links": "U = exp(i eps X), plaquette 0.59, seed %d" % w["link_seed"],
            "precision": precision_text(w, j1_of(w, args)),
            "p": "one p per batch: Eq. popt with z_min, z_max of A estimated as the extremes over the "
                 "batch's H_k (power / inverse iteration)",
            "graph": True, "parallelism": "replicas" if args.gpus > 1 else "single",
            "batches_in_flight": args.inflight, "nested_levels": [w["ell"], *w.get("nest", ())],
            "l2": "working set (Krylov basis %.1f GB per batch) larger than L2" % (
                12 * w["n_rhs"] * np.prod(w["dims"]) * w["k"] * 16 / 1e9)}


def new_context(nk, w, U, j1, shape=None, n_rhs=None, flags=0):
    c = nk.Context(w["dims"])
    c.load_links(U)
    c.set_mu_mw(w["mu"], w["m_w"])
    c.set_precision(w.get("j0", -1))
    c.set_df_recurrence(j1)
    c.set_nesting(w.get("nest", ()))
    if shape is not None:
        c.set_launch(n_rhs, flags, *shape)
    return c


def timed_batches(nk, torch, ctxs, b_dev, ys, streams, w, flags, steps, warmup):
    """warmup then `steps` whole batched solves, len(ctxs) in flight on their own
    streams (NK_ASYNC + nk_wait); returns (ms, launches) of the timed region
    (CUDA events on the current stream, which waits for every stream)."""
    n_rhs, k, ell = w["n_rhs"], w["k"], w["ell"]
    inflight = len(ctxs)
    for _ in range(warmup):
        for c_, y_ in zip(ctxs, ys):
            c_.sign_apply_dev(b_dev, y_, n_rhs, k, ell, flags=flags)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s_ in streams:
        s_.wait_stream(stream)
    launches = 0
    for i in range(steps):
        c_ = ctxs[i % inflight]
        if inflight > 1:
            if i >= inflight:
                st, _ = c_.wait()
                launches += st["launches"]
            c_.sign_apply_dev(b_dev, ys[i % inflight], n_rhs, k, ell, flags=flags | nk.NK_ASYNC,
                              stream=streams[i % inflight])
        else:
            st, _ = c_.sign_apply_dev(b_dev, ys[0], n_rhs, k, ell, flags=flags)
            launches += st["launches"]
    if inflight > 1:
        for c_ in ctxs:
            st, _ = c_.wait()
            launches += st["launches"]
        for s_ in streams:
            stream.wait_stream(s_)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), launches


def rel_errs(y, ref):
    return [float(np.linalg.norm(y[i] - ref[i]) / np.linalg.norm(ref[i])) for i in range(len(ref))]


def stencil_roofline(nk, torch, peaks):
    """The solver's FP32 stencil kernel alone (12 RHS of A and 12 of A^dagger
    per launch, FP32 vectors in and out) on 16^3 x 32, a lattice whose vectors
    are larger than L2: achieved algorithmic GB/s from CUDA events around
    repeated launches on the launch stream (nk_stencil32_dev), against the
    measured HBM copy bandwidth.  Algorithmic bytes per launch (each array
    moved once): FP32 links 288 B/site + per vector FP32 input 96 B and FP32
    output 96 B per site."""
    import inputs
    dims = STENCIL_DIMS
    ctx = nk.Context(dims)
    ctx.load_links(inputs.su3_links(dims, 105)[0])
    ctx.set_mu_mw(0.2, -2.0)
    V = int(np.prod(dims))
    n = 12
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(2 * n * 24 * V, dtype=torch.float32, device="cuda", generator=g)
    out = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        ctx.stencil32_dev(x, out, n)
    torch.cuda.synchronize()
    reps = 20
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):     # input and output (302 MB each) are larger than L2
        ctx.stencil32_dev(x, out, n)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    total = V * (288 + 2 * n * 192)
    gbs = total / (ms * 1e-3) / 1e9
    ctx.close()
    return {"kernel": "k_stencil32 (FP32 Wilson stencil, 12 RHS of A + 12 of A^dagger per launch, links "
                      "loaded once per site block for all 24 vectors)",
            "lattice": "16x16x16x32", "bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs"),
            "unit": "GB/s", "frac": gbs / peaks.get("hbm_gbs", 6800.0), "ms_per_launch": ms,
            "bytes_per_launch": total, "launches": reps, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": profiled_traffic("k_stencil32@16x16x16x32")}


def dominant_roofline(dom, tc, nc, w, peaks, sm_mhz):
    """Roofline entry for the kernel class with the largest device time.

    Algorithmic work per launch, n_rhs sources, two-sided (Hermitian in
    parentheses); each array moved once, each flop of the method counted once:
      step2 (the FP64 recurrence kernels k_step1 and k_step2, one launch of
             each per FP32 step): step 1 r = s - c1 q_{j-1}, l = t - c1' p_{j-1},
             H(j,j) += p_j^dag r; step 2 r -= c3 q_j, l -= c4 p_j,
             delta += r^dag l: 24 (8) FP64 flops per element in either kernel
             -- FP64 ALU, peak the nominal 1.25 TFLOP/s; bytes per element:
             step 1 loads s, t (FP32) and q_{j-1}, p_{j-1}, p_j, stores r, l
             (96 (56) B), step 2 loads q_j, r, p_j, l, stores r, l and their
             FP32 copies (112 (56) B);
      dslash (the multi-RHS FP32 stencil of the FP32 steps): links 288 B per
             site plus 96 B in and 96 B out per site and vector -- HBM;
      dslash_df: the two-float stencil, 1320 flops per site and vector;
             a two-float multiply-add costs 12 FP32 lane operations for its
             2 flops, so its ALU peak is 152 x 128 x f_SM / 6;
      lift (FP64): y += c_j q_j over k columns: 8 FP64 flops per element and
             column -- FP64 ALU;
      inner / rhi: FP64 ALU, latency bound on few SMs (not modelled).
    """
    V = int(np.prod(w["dims"]))
    N = 12 * V
    n_rhs = w["n_rhs"]
    two = w["mu"] != 0.0
    nv = (2 if two else 1) * n_rhs
    ms = tc[dom] / max(1, nc[dom])
    hbm = peaks.get("hbm_gbs", 6800.0)

    def alu64(kernel, flops, extra=None):
        tf = flops / (ms * 1e-3) / 1e12
        r = {"kernel": kernel, "bound": "alu", "achieved": tf, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
             "frac": tf / FP64_PEAK_TFLOPS, "ms_per_launch": ms, "flops_per_launch": flops,
             "peak_derivation": "nominal dense FP64 rate of GB300 (1.25 TFLOP/s, 152 SMs); a DFMA throughput "
                                "test on this pool measured 0.59-0.63 T DFMA/s, i.e. the same"}
        r.update(extra or {})
        return r

    if dom == "step2":
        t1, t2 = profiled_traffic("k_step1"), profiled_traffic("k_step2")   # the FP32-step pair
        return alu64("k_step1 / k_step2 (FP64 recurrence, operands staged by bulk copies)",
                     (24 if two else 8) * N * n_rhs,
                     {"traffic": (t1 + t2) / 2 if (t1 is not None and t2 is not None) else None,
                      "algorithmic_bytes_per_launch": (104 if two else 56) * N * n_rhs})
    if dom == "dslash":
        nbytes = (288.0 + nv * 192.0) * V
        gbs = nbytes / (ms * 1e-3) / 1e9
        return {"kernel": "k_stencil32 (multi-RHS FP32 stencil of the FP32 steps)", "bound": "hbm",
                "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "ms_per_launch": ms,
                "bytes_per_launch": nbytes, "traffic": profiled_traffic("k_stencil32@10x10x10x10")}
    if dom == "lift":
        return alu64("k_lift (FP64)", 8.0 * N * n_rhs * w["k"], {"traffic": None})
    if dom == "dslash_df":
        flops = 1320.0 * V * nv
        tf = flops / (ms * 1e-3) / 1e12
        peak = 152 * 128 * (sm_mhz or 2070.0) * 1e6 / 6.0 / 1e12
        return {"kernel": "k_stencil_df (multi-RHS two-float stencil)", "bound": "alu",
                "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                "traffic": profiled_traffic("k_stencil_df"), "ms_per_launch": ms, "flops_per_launch": flops,
                "peak_derivation": "FP32 FMA pipe 152 x 128 lanes x f_SM over the 6 FP32 lane operations per "
                                   "two-float flop of a two-float multiply-add (TwoProd by FMA, its two cross "
                                   "terms, TwoSum and the trailing sum: 12 operations for 2 flops)"}
    return {"kernel": dom, "bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": None, "traffic": None, "ms_per_launch": ms, "hbm_gbs": hbm}


def learned_arm(nk, torch, ctx, b_dev, w, flags):
    """Adaptive k (tol = TOL, NK_ADAPT_STEP = 64) on the batch, (a) from the
    default start NK_ADAPT_FIRST(l) with the workload's l, (b) from the
    predicted sizes: the predictor (predictor_weights.npz, trained on runs of
    the method) gives (k, l) from the features of source 0; checks start at
    k_pred - 128 with l = 1.5 l_pred.  Solves/s count the sources that the
    adaptive stop accepted (NK_OK); each arm is timed on a warm repeat."""
    from paper_0912_4457_gb300 import predictor
    n_rhs = w["n_rhs"]
    y = torch.zeros_like(b_dev)
    k_max = predictor.K_MAX
    out = {}
    m = predictor.load_model()
    t0 = time.perf_counter()
    k_pred, l_pred = ctx.predict_sizes(m, b_dev[:1].contiguous(), k_max)
    t_pred = time.perf_counter() - t0
    l_use = min(256, k_pred, 2 * int(np.ceil(0.75 * l_pred)))
    for name, start, ell in (("adaptive_default", 0, w["ell"]), ("adaptive_predicted", max(64, k_pred - 128), l_use)):
        ctx.set_adapt_start(start)
        try:
            for rep in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, rc = ctx.sign_apply_dev(b_dev, y, n_rhs, k_max, ell, tol=TOL, flags=flags, check=False)
                torch.cuda.synchronize()
                wall = time.perf_counter() - t0
        finally:
            ctx.set_adapt_start(0)
        ok = sum(1 for s in st["status"] if s == 0)
        out[name] = {"value": ok / wall, "unit": "solves/s", "wall_ms": 1e3 * wall, "device_ms": st["t_total_ms"],
                     "checks": st["checks"], "k_rhs": st["k_rhs"], "ell": ell, "start": start or None, "rc": rc,
                     "y": y.cpu().numpy()}
    out["prediction"] = {"k": k_pred, "ell": l_pred, "ms": 1e3 * t_pred}
    m.close()
    return out


def multilevel_arm(nk, torch, ctx, b_dev, w, flags, y_ref):
    """Multi-level nesting (Sec. 4.5) on the batch of the workload: one level
    (l = w["ell"]) against deeper chains l -> l_2 -> ... (RHi on the deepest
    Ritz matrix).  One batch at a time (graph, CUDA events around two warm
    solves); the inner part's device time from NK_PROFILE (classes inner +
    rhi); every source against the FP64 reference, so a chain too short for
    the tolerance shows as such."""
    n_rhs, k, ell = w["n_rhs"], w["k"], w["ell"]
    y = torch.zeros_like(b_dev)
    stream = torch.cuda.current_stream()
    out = {}
    for levels in ((), (96,), (64,), (64, 16), (32, 8)):
        name = "levels_" + "_".join(str(v) for v in (ell, *levels))
        ctx.set_nesting(levels)
        try:
            ctx.sign_apply_dev(b_dev, y, n_rhs, k, ell, flags=flags)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                ctx.sign_apply_dev(b_dev, y, n_rhs, k, ell, flags=flags)
            e1.record(stream)
            torch.cuda.synchronize()
            err = rel_errs(y.cpu().numpy(), y_ref)
            st, _ = ctx.sign_apply_dev(b_dev, y, n_rhs, k, ell, flags=flags | nk.NK_PROFILE)
            torch.cuda.synchronize()
        finally:
            ctx.set_nesting(w.get("nest", ()))
        ms = e0.elapsed_time(e1) / 2
        ok = sum(1 for e in err if e <= TOL)
        out[name] = {"ells": [ell, *levels], "ms_per_batch": ms, "solves_per_s_one_batch": ok / (ms * 1e-3),
                     "inner_ms": st["t_class_ms"]["inner"] + st["t_class_ms"]["rhi"],
                     "rhi_iters_max": max(st["rhi_iters"]), "max_rel_err_vs_fp64_reference": max(err)}
    return out


DEFLATION_CASE = dict(dims=(6, 6, 6, 6), mu=0.0, m_w=-2.0, link_seed=102, eig_seed=203, k_eig=2400, m=16,
                      tol_eig=1e-10, k_max=1536, ell=128, k_fixed=256, k_ref=1536, ell_ref=256)


def deflation_arm(nk, torch):
    """LR deflation (App. C steps 1 and 6) with its eigenpairs from the
    device eigensolver (nk_eigs_smallest: k_eig FP64 Lanczos steps from a
    Gaussian vector, the m pairs of smallest |lambda| with residual <=
    tol_eig; a one-off initialisation, timed separately).  Then the 12
    spin-colour point sources at 6^4, mu = 0, FP64, adaptive k (tol = TOL)
    without and with the deflation: k reached per source, device time, and
    every source against the undeflated FP64 solve at k = 1536, l = 256; and
    the error of both at a fixed smaller k (k_fixed)."""
    import inputs
    c = DEFLATION_CASE
    U, _ = inputs.su3_links(c["dims"], c["link_seed"])
    flags = nk.NK_FP64 | nk.NK_SHARED_P
    ctx = nk.Context(c["dims"])
    try:
        ctx.load_links(U)
        ctx.set_mu_mw(c["mu"], c["m_w"])
        t0 = time.perf_counter()
        lam, R, L, res, rc_e = ctx.eigs_smallest(inputs.gaussian_sources(c["dims"], c["eig_seed"])[0], c["k_eig"],
                                                 c["m"], tol=c["tol_eig"], check=False)
        t_eig = time.perf_counter() - t0
        b_dev = torch.from_numpy(np.ascontiguousarray(inputs.point_sources(c["dims"]))).cuda()
        n = b_dev.shape[0]
        yref = torch.zeros_like(b_dev)
        ctx.sign_apply_dev(b_dev, yref, n, c["k_ref"], c["ell_ref"], flags=flags)
        torch.cuda.synchronize()
        y_ref = yref.cpu().numpy()
        out = {"lattice": "x".join(map(str, c["dims"])), "mu": c["mu"], "tol": TOL, "k_fixed": c["k_fixed"],
               "eigensolver": {"k": c["k_eig"], "m": c["m"], "tol": c["tol_eig"], "rc": rc_e, "found": len(lam),
                               "max_residual": float(max(res)) if len(res) else None,
                               "abs_lambda": [float(abs(x)) for x in lam], "wall_s": t_eig}}
        y = torch.zeros_like(b_dev)
        for name, pairs in (("undeflated", None), ("deflated", (lam, R, L) if len(lam) else None)):
            if name == "deflated" and pairs is None:
                break
            ctx.set_deflation(*(pairs or (None,)))
            for _ in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, rc = ctx.sign_apply_dev(b_dev, y, n, c["k_max"], c["ell"], tol=TOL, flags=flags, check=False)
                torch.cuda.synchronize()
                wall = time.perf_counter() - t0
            err = rel_errs(y.cpu().numpy(), y_ref)
            ctx.sign_apply_dev(b_dev, y, n, c["k_fixed"], c["ell"], flags=flags)
            torch.cuda.synchronize()
            err_fixed = rel_errs(y.cpu().numpy(), y_ref)
            out[name] = {"k_rhs": st["k_rhs"], "checks": st["checks"], "device_ms": st["t_total_ms"],
                         "wall_ms": 1e3 * wall, "rc": rc, "defl_m": st["defl_m"], "defl_gap": st["defl_gap"],
                         "max_rel_err_vs_fp64_reference": max(err),
                         "solves_meeting_tol": sum(1 for e in err if e <= TOL),
                         "max_rel_err_at_k_fixed": max(err_fixed)}
        ctx.set_deflation(None)
    finally:
        ctx.close()
    return out


OVERLAP_CASE = dict(dims=(6, 6, 6, 6), mu=0.3, m_w=-2.0, link_seed=102, source_seed=202, k=512, ell=128,
                    mass=0.05, tol_cg=1e-8, maxit=400)


def overlap_arm(nk):
    """Overlap inversion x = (D_ov(mu) + mass)^-1 b (CG on the normal
    equations, every iteration one sign evaluation of A(mu) and one of
    A(-mu)) on the 6^4, mu = 0.3 configuration's sizes (k = 512, l = 128,
    FP64), one Gaussian source; the true residual |b - (D_ov + mass) x| / |b|
    from one more overlap application."""
    import inputs
    c = OVERLAP_CASE
    U, _ = inputs.su3_links(c["dims"], c["link_seed"])
    b = inputs.gaussian_sources(c["dims"], c["source_seed"])
    ctx = nk.Context(c["dims"])
    try:
        ctx.load_links(U)
        ctx.set_mu_mw(c["mu"], c["m_w"])
        t0 = time.perf_counter()
        x, its, res, rc = ctx.overlap_solve(b, c["k"], c["ell"], mass=c["mass"], tol_cg=c["tol_cg"],
                                            maxit=c["maxit"], flags=nk.NK_FP64, check=False)
        wall = time.perf_counter() - t0
        dx, _, _ = ctx.overlap_apply(x, c["k"], c["ell"], flags=nk.NK_FP64)
        true_res = float(np.linalg.norm(b - dx - c["mass"] * x) / np.linalg.norm(b))
    finally:
        ctx.close()
    return {"lattice": "x".join(map(str, c["dims"])), "mu": c["mu"], "k": c["k"], "ell": c["ell"],
            "mass": c["mass"], "tol_cg": c["tol_cg"], "rc": rc, "cg_iterations": int(its[0]),
            "normal_eq_rel_residual": float(res[0]), "true_rel_residual": true_res, "wall_s": wall,
            "ms_per_iteration": 1e3 * wall / max(1, int(its[0])),
            "what": "CG on M^dagger M x = M^dagger b, M = D_ov(mu) + mass, two FP64 sign evaluations per "
                    "iteration, one Gaussian source"}


def run_gpu(args, w, rank, world, local_rank):
    import multiprocessing as mp
    import torch
    import paper_0912_4457_gb300 as nk
    from paper_0912_4457_gb300 import build as nkbuild
    if not os.path.exists(nkbuild.LIB) or not nkbuild.up_to_date():
        if rank == 0:
            nkbuild.build()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
    dist = None
    if world > 1:
        import torch.distributed as dist
    peaks = measured_peaks()
    U, b_host = make_inputs(w)
    n_rhs, k, ell = w["n_rhs"], w["k"], w["ell"]
    j1 = j1_of(w, args)
    flags = (nk.NK_MIXED if w["mixed"] else nk.NK_FP64) | nk.NK_SHARED_P
    torch.cuda.set_device(local_rank)
    ctx = new_context(nk, w, U, j1)
    # launch shape of the outer recurrence: timed on 16 synthetic steps, kept
    shape, tune_ms = ctx.autotune(n_rhs, flags, args.tune_cache)
    b_dev = torch.from_numpy(np.ascontiguousarray(b_host)).cuda()
    st0, _ = ctx.sign_apply_dev(b_dev, torch.zeros_like(b_dev), n_rhs, k, ell, flags=flags)
    torch.cuda.synchronize()
    p_batch = float(st0["p"][0])
    # the oracle on source 0 (same k, l, p), in a spawned process beside the GPU work
    pool = None
    if rank == 0 and not args.quick:
        pool = mp.get_context("spawn").Pool(1)
        oracle_job = pool.apply_async(_oracle_solve, ((U, w["dims"], w["mu"], w["m_w"], b_host[0], k, ell, p_batch,
                                                        tuple(w.get("nest", ()))),))

    # ---- headline: fixed k, batches in flight -----------------------------------
    inflight = max(1, args.inflight)
    ctxs = [ctx] + [new_context(nk, w, U, j1, shape, n_rhs, flags) for _ in range(1, inflight)]
    ys = [torch.zeros_like(b_dev) for _ in range(inflight)]
    streams = [torch.cuda.Stream() for _ in range(inflight)]
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    ms_raw, launches = timed_batches(nk, torch, ctxs, b_dev, ys, streams, w, flags, args.steps, args.warmup)
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ms_raw, dist)
    y = ys[(args.steps - 1) % inflight].cpu().numpy()
    # the two-float recurrence (a second, labelled line of the same workload)
    df = None
    if not args.quick:
        for c_ in ctxs:
            c_.set_df_recurrence(0)
        ms_df, _ = timed_batches(nk, torch, ctxs, b_dev, ys, streams, w, flags, max(4, args.steps // 2), 1)
        y_df = ys[(max(4, args.steps // 2) - 1) % inflight].cpu().numpy()
        for c_ in ctxs:
            c_.set_df_recurrence(j1)
        df = {"ms_per_step": ms_df / max(4, args.steps // 2), "y": y_df}
    for c_ in ctxs[1:]:
        c_.close()
    # latency of one batch with nothing else in flight
    l0 = torch.cuda.Event(enable_timing=True)
    l1 = torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    y_dev = torch.zeros_like(b_dev)
    l0.record(stream)
    for _ in range(2):
        ctx.sign_apply_dev(b_dev, y_dev, n_rhs, k, ell, flags=flags)
    l1.record(stream)
    torch.cuda.synchronize()
    latency_ms = l0.elapsed_time(l1) / 2

    # ---- e2e: pinned host buffers through the host-pointer C entry point -----------
    b_pin = torch.from_numpy(np.ascontiguousarray(b_host)).pin_memory()
    y_pin = torch.zeros_like(b_pin).pin_memory()
    bp, yp = b_pin.numpy(), y_pin.numpy()
    _lib_host_solve(ctx, bp, yp, k, ell, flags)
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        _lib_host_solve(ctx, bp, yp, k, ell, flags)
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    # ---- comparator named by the metric: all-FP64 nested method, one source per solve
    b1 = b_dev[:1].contiguous()
    y1 = torch.zeros_like(b1)
    ctx.sign_apply_dev(b1, y1, 1, k, ell, p=p_batch, flags=nk.NK_FP64)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    nrep = 2
    f0.record(stream)
    for _ in range(nrep):
        ctx.sign_apply_dev(b1, y1, 1, k, ell, p=p_batch, flags=nk.NK_FP64)
    f1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = f0.elapsed_time(f1) / nrep
    y_fp64 = y1.cpu().numpy()[0]

    # ---- converged FP64 reference for every source (GPU, larger k and l) ----------
    yref = torch.zeros_like(b_dev)
    ctx.sign_apply_dev(b_dev, yref, n_rhs, w["k_ref"], w["ell_ref"], flags=nk.NK_FP64 | nk.NK_SHARED_P)
    torch.cuda.synchronize()
    y_ref = yref.cpu().numpy()
    err_ref = rel_errs(y, y_ref)

    # ---- per-kernel-class device times (NK_PROFILE: CUDA events around each launch)
    stp, _ = ctx.sign_apply_dev(b_dev, y_dev, n_rhs, k, ell, flags=flags | nk.NK_PROFILE)
    torch.cuda.synchronize()
    learned = None if args.quick else learned_arm(nk, torch, ctx, b_dev, w, flags)
    multilevel = None if args.quick else multilevel_arm(nk, torch, ctx, b_dev, w, flags, y_ref)
    if rank != 0:
        ctx.close()
        return 0
    sten = stencil_roofline(nk, torch, peaks)

    # ---- accuracy: every source against the FP64 reference; source 0 against the oracle
    err0 = None
    t_or = None
    if pool is not None:
        y_or, t_or = oracle_job.get()
        pool.close()
        pool.join()
        err0 = float(np.linalg.norm(y[0] - y_or) / np.linalg.norm(y_or))
        err_fp64_or = float(np.linalg.norm(y_fp64 - y_or) / np.linalg.norm(y_or))
    ok = sum(1 for e in err_ref if e <= TOL)
    if err0 is not None and err0 > TOL:
        ok = 0
    value = whole_job_value(ok, args.steps, ms, world)
    e2e_value = ok / e2e_s
    tc = stp["t_class_ms"]
    nc = stp["n_class"]
    tot = sum(tc.values())
    share = {kk: (tc[kk] / tot if tot else 0.0) for kk in tc}
    dom = max(tc, key=lambda kk: tc[kk])
    roof = dominant_roofline(dom, tc, nc, w, peaks, clocks.get("sm_mhz"))
    fp64_ok = float(np.linalg.norm(y_fp64 - y_ref[0]) / np.linalg.norm(y_ref[0])) <= TOL
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "latency_ms_one_batch": latency_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": config_of(w, args),
        "accuracy": {"tol": TOL, "solves_meeting_tol": ok,
                     "rel_err_vs_fp64_reference": err_ref,
                     "fp64_reference": "the same batch all in FP64 at k = %d, l = %d (converged: k = 1024 is "
                                       "within 1e-11 of it)" % (w["k_ref"], w["ell_ref"]),
                     "rel_err_vs_oracle_src0": err0,
                     "oracle": "nested oracle (numpy FP64) on source 0, same k, l and p"},
        "e2e": {"value": e2e_value, "unit": "solves/s",
                "h2d_bytes_per_step": int(b_host.nbytes), "d2h_bytes_per_step": int(b_host.nbytes)},
        "fp64_plain": {"value": (1.0 / (fp64_ms * 1e-3)) if fp64_ok else 0.0, "unit": "solves/s",
                       "ms_per_solve": fp64_ms,
                       "rel_err_vs_fp64_reference_src0": float(np.linalg.norm(y_fp64 - y_ref[0]) /
                                                               np.linalg.norm(y_ref[0])),
                       "what": "same method, all FP64 (stencil and recurrence), one source per solve, same k, "
                               "l and p, same GPU"},
        "speedup_vs_fp64_plain": (value / world) / (1.0 / (fp64_ms * 1e-3)),
        "gpu_launches": launches,
        "launch_shape": {"stencil_threads": shape[0], "stencil_order": shape[1], "step2_blocks": shape[2],
                         "early_threads": shape[3], "early_order": shape[4], "stencil_split": shape[5],
                         "early_split": shape[6], "autotune_ms_per_outer_step": tune_ms},
        "rhi_iters": stp["rhi_iters"],
        "kernel_class_ms": {kk: round(v, 3) for kk, v in tc.items()},
        "kernel_time_share": {kk: round(v, 4) for kk, v in share.items()},
        "roofline": roof,
        "stencil_roofline": sten,
        "clocks": clocks,
    }
    if df is not None:
        e_df = rel_errs(df["y"], y_ref)
        ok_df = sum(1 for e in e_df if e <= TOL)
        line["two_float_recurrence"] = {
            "value": whole_job_value(ok_df, 1, df["ms_per_step"], world), "unit": "solves/s",
            "ms_per_step": df["ms_per_step"], "max_rel_err_vs_fp64_reference": max(e_df),
            "what": "the same workload with the recurrence in two-float (about 48-bit) arithmetic from step 0 "
                    "(nk_set_df_recurrence(0)) and a two-float lift; not the headline (narrower than FP64)"}
    if learned is not None:
        blk = {}
        for name in ("adaptive_default", "adaptive_predicted"):
            r = dict(learned[name])
            e = rel_errs(r.pop("y"), y_ref)
            r["max_rel_err_vs_fp64_reference"] = max(e)
            blk[name] = r
        blk["prediction"] = learned["prediction"]
        blk["fixed_k"] = {"value": value, "k": k, "ell": ell}
        line["learned"] = blk
    if multilevel is not None:
        line["multilevel"] = multilevel
    if not args.quick:
        line["deflation"] = deflation_arm(nk, torch)
        line["overlap_solve"] = overlap_arm(nk)
    if pool is not None:
        one, allc = cpu_baselines(w)
        line["cpu_baseline"] = one
        line["cpu_baseline_all_cores"] = allc
        line["accuracy"]["rel_err_fp64_plain_vs_oracle_src0"] = err_fp64_or
        line["accuracy"]["oracle_seconds"] = t_or
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
    ctx = new_context(nk, w, U, j1_of(w, args))
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


def run_stencil(args):
    """--mode stencil: --warmup + 1 launches of the multi-RHS FP32 stencil alone
    (nk_stencil32_dev: 12 RHS of A and 12 of A^dagger) on 16^3 x 32, for ncu
    captures of that kernel; prints its CUDA-event time per launch to stderr."""
    import torch
    import inputs
    import paper_0912_4457_gb300 as nk
    dims = STENCIL_DIMS
    ctx = nk.Context(dims)
    ctx.load_links(inputs.su3_links(dims, 105)[0])
    ctx.set_mu_mw(0.2, -2.0)
    V = int(np.prod(dims))
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(2 * 12 * 24 * V, dtype=torch.float32, device="cuda", generator=g)
    out = torch.empty_like(x)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for i in range(args.warmup + 1):
        e0.record()
        ctx.stencil32_dev(x, out, 12)
        e1.record()
    torch.cuda.synchronize()
    print("stencil32 16x16x16x32, 24 vectors: %.3f ms per launch" % e0.elapsed_time(e1), file=sys.stderr)
    ctx.close()
    return 0


def run_rows(args, w):
    """--mode rows: the multi-level, deflation and overlap-inversion blocks of
    the bench line alone (multi-level on the workload's batch against its FP64
    reference), printed as one JSON line."""
    import torch
    import paper_0912_4457_gb300 as nk
    U, b_host = make_inputs(w)
    n_rhs = w["n_rhs"]
    flags = (nk.NK_MIXED if w["mixed"] else nk.NK_FP64) | nk.NK_SHARED_P
    ctx = new_context(nk, w, U, j1_of(w, args))
    try:
        ctx.autotune(n_rhs, flags, args.tune_cache)
        b_dev = torch.from_numpy(np.ascontiguousarray(b_host)).cuda()
        yref = torch.zeros_like(b_dev)
        ctx.sign_apply_dev(b_dev, yref, n_rhs, w["k_ref"], w["ell_ref"], flags=nk.NK_FP64 | nk.NK_SHARED_P)
        torch.cuda.synchronize()
        multilevel = multilevel_arm(nk, torch, ctx, b_dev, w, flags, yref.cpu().numpy())
    finally:
        ctx.close()
    print(json.dumps({"multilevel": multilevel, "deflation": deflation_arm(nk, torch),
                      "overlap_solve": overlap_arm(nk)}))
    return 0


def _lib_host_solve(ctx, bp, yp, k, ell, flags):
    import ctypes
    from paper_0912_4457_gb300 import nksign
    st = nksign.NkStats()
    rc = ctx._lib.nk_sign_apply(ctx.h, nksign._dptr(bp.view(np.float64)), bp.shape[0], int(k), int(ell), 0.0,
                                0.0, int(flags), nksign._dptr(yp.view(np.float64)), ctypes.byref(st))
    ctx._check(rc)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--mode", choices=["bench", "ncu", "stencil", "rows"], default="bench",
                    help="ncu: run --warmup solves and then one solve kernel by kernel (no graph, no oracle, "
                         "no output line), for launch lists and captures under ncu; stencil: --warmup + 1 "
                         "launches of the FP32 stencil alone on 16^3 x 32; rows: only the multi-level, deflation "
                         "and overlap-inversion blocks of the bench line, printed as one JSON line")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--ncu-k", type=int, default=0, help="--mode ncu: outer steps (0: the workload's k)")
    ap.add_argument("--j1", type=int, default=None,
                    help="first outer step with a two-float recurrence (default: the workload's; -1: none)")
    ap.add_argument("--inflight", type=int, default=4,
                    help="batches in flight (contexts on their own streams); 1: one synchronous solve per step")
    ap.add_argument("--tune-cache", default=None,
                    help="launch-shape cache file (read if it has the workload's shape, else written)")
    ap.add_argument("--nest", default="",
                    help="comma-separated sizes l_2, l_3, ... of nested levels below l (Sec. 4.5), or 'none' "
                         "for one level (default: the workload's)")
    ap.add_argument("--quick", action="store_true",
                    help="headline only: no oracle, CPU baselines, two-float line or learned arm")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    w = dict(WORKLOADS[args.workload])
    if args.nest == "none":
        w["nest"] = ()
    elif args.nest:
        w["nest"] = tuple(int(v) for v in args.nest.split(","))
    if args.impl == "reference":
        return run_reference(args, w, rank)
    if args.mode == "ncu":
        return run_ncu(args, w)
    if args.mode == "stencil":
        return run_stencil(args)
    if args.mode == "rows":
        return run_rows(args, w)
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
