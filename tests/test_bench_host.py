"""Host logic of bench.py (no GPU): the workload's schedule, the roofline
arithmetic, the throughput formula and the committed ncu traffic figures."""
import argparse

import numpy as np
import pytest

import bench


def _args(**kw):
    a = argparse.Namespace(j1=None, inflight=4, gpus=1, workload=bench.DEFAULT_WORKLOAD)
    for k, v in kw.items():
        setattr(a, k, v)
    return a


def test_default_workload_is_the_largest_single_gpu_config():
    """10^4, mu = 0.2, 12 point sources, FP32 stencil after j0 and an FP64 recurrence."""
    w = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert w["dims"] == (10, 10, 10, 10) and w["mu"] == 0.2 and w["n_rhs"] == 12
    assert w["mixed"] and bench.j1_of(w, _args()) == -1
    assert w["k_ref"] > w["k"] and w["ell_ref"] >= w["ell"]


def test_df_recurrence_start_of_the_workload():
    w = dict(bench.WORKLOADS[bench.DEFAULT_WORKLOAD])
    assert bench.j1_of(w, _args()) == -1                      # FP64 recurrence throughout
    assert bench.j1_of(w, _args(j1=-5)) == -1
    assert bench.j1_of(w, _args(j1=0)) == 0
    assert bench.j1_of(w, _args(j1=300)) == 300


def test_whole_job_value_counts_every_rank():
    # 12 solves per step, 24 steps, 1 s: 288 solves/s per rank
    assert bench.whole_job_value(12, 24, 1000.0, 1) == pytest.approx(288.0)
    assert bench.whole_job_value(12, 24, 1000.0, 4) == pytest.approx(4 * 288.0)


def test_roofline_of_the_fp64_step2():
    """Two-sided step 2: r -= c3 q, l -= c4 p, delta += r^dag l, 24 FP64 flops
    per element against the nominal FP64 rate."""
    w = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    N = 12 * int(np.prod(w["dims"]))
    tc, nc = {"step2": 5.0}, {"step2": 100}            # 50 us per launch
    r = bench.dominant_roofline("step2", tc, nc, w, {"hbm_gbs": 6000.0}, 2070.0)
    flops = 24.0 * N * w["n_rhs"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["flops_per_launch"] == pytest.approx(flops)
    assert r["achieved"] == pytest.approx(flops / 50e-6 / 1e12)
    assert r["peak"] == pytest.approx(bench.FP64_PEAK_TFLOPS)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_roofline_of_the_two_float_stencil():
    w = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    V = int(np.prod(w["dims"]))
    tc, nc = {"dslash_df": 25.6}, {"dslash_df": 256}   # 100 us per launch
    r = bench.dominant_roofline("dslash_df", tc, nc, w, {"hbm_gbs": 6000.0}, 2070.0)
    flops = 1320.0 * V * 2 * w["n_rhs"]                   # two-sided: A and A^dagger
    assert r["flops_per_launch"] == pytest.approx(flops)
    assert r["achieved"] == pytest.approx(flops / 1e-4 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2070e6 / 6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_committed_profiles_give_the_traffic_of_the_outer_kernels():
    for kernel in ("k_step1", "k_step2", "k_stencil_df", "k_stencil32@10x10x10x10", "k_stencil32@16x16x16x32"):
        assert bench.profiled_traffic(kernel) is not None, kernel
    assert bench.profiled_traffic("no_such_kernel") is None


def test_config_names_the_workload_and_its_schedule():
    w = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    c = bench.config_of(w, _args())
    assert c["workload"] == bench.DEFAULT_WORKLOAD
    assert c["lattice"] == "x".join(str(d) for d in w["dims"])
    assert c["batches_in_flight"] == 4
    assert c["k"] == w["k"] and c["ell"] == w["ell"] and c["n_rhs"] == w["n_rhs"]
    assert "recurrence" in c["precision"] and "FP64" in c["precision"]
    assert "two-float (about 48-bit) from it on" in bench.config_of(w, _args(j1=0))["precision"]


def test_nested_levels_of_the_workload_and_its_record():
    """The bench workload nests l_2 = 64 below l = 128 (Sec. 4.5); the line's
    config records the chain, and every level is even and no larger than the
    one above."""
    w = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    chain = [w["ell"], *w.get("nest", ())]
    assert chain == [128, 64]
    assert all(v % 2 == 0 and v >= 2 for v in chain) and chain == sorted(chain, reverse=True)
    cfg = bench.config_of(w, _args())
    assert cfg["nested_levels"] == chain


def test_next_row_cases_are_valid_calls():
    """The deflation and overlap blocks call the library with arguments its
    header accepts: eigensolver k even and >= 2 m + 2, m <= 256; solve sizes
    even, l <= k <= 1536, l <= 256; the fixed-k comparison below the
    adaptive maximum."""
    d = bench.DEFLATION_CASE
    assert d["k_eig"] % 2 == 0 and d["k_eig"] >= 2 * d["m"] + 2 and 1 <= d["m"] <= 256
    for k, ell in ((d["k_max"], d["ell"]), (d["k_ref"], d["ell_ref"]), (d["k_fixed"], d["ell"])):
        assert k % 2 == 0 and ell % 2 == 0 and 2 <= ell <= min(k, 256) and k <= 1536
    assert d["k_fixed"] < d["k_max"] and d["tol_eig"] > 0
    o = bench.OVERLAP_CASE
    assert o["k"] % 2 == 0 and o["ell"] % 2 == 0 and o["ell"] <= o["k"] <= 1536 and o["mass"] >= 0


def test_reference_arm_line(monkeypatch, capsys):
    """--impl reference: the oracle's outer recurrence on a bounded sample,
    one JSON line with the contract's keys (run here on a 4^4 stand-in of the
    workload with a one-second budget)."""
    import json
    w = dict(bench.WORKLOADS[bench.DEFAULT_WORKLOAD], dims=(4, 4, 4, 4), k=64)
    monkeypatch.setattr(bench, "REF_BUDGET_S", 1.0)
    args = _args(steps=2, warmup=1)
    assert bench.run_reference(args, w, 0) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "solves/s"
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == bench.DEFAULT_WORKLOAD
    # other ranks print nothing
    assert bench.run_reference(args, w, 1) == 0 and capsys.readouterr().out == ""
