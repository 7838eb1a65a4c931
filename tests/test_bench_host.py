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


def test_df_recurrence_start_of_the_workload():
    w = dict(bench.WORKLOADS[bench.DEFAULT_WORKLOAD])
    want = w["j0"] if w.get("j1", -1) < 0 else min(w["j1"], w["j0"])
    assert bench.j1_of(w, _args()) == want
    assert bench.j1_of(w, _args(j1=-1)) == w["j0"]            # < 0: the FP32 switch
    assert bench.j1_of(w, _args(j1=10 * w["j0"])) == w["j0"]  # past j0 acts as j0
    assert bench.j1_of(w, _args(j1=0)) == 0


def test_whole_job_value_counts_every_rank():
    # 12 solves per step, 24 steps, 1 s: 288 solves/s per rank
    assert bench.whole_job_value(12, 24, 1000.0, 1) == pytest.approx(288.0)
    assert bench.whole_job_value(12, 24, 1000.0, 4) == pytest.approx(4 * 288.0)


def test_roofline_of_the_two_float_stencil():
    w = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    V = int(np.prod(w["dims"]))
    tc, nc = {"dslash_df": 25.6}, {"dslash_df": 256}   # 100 us per launch
    r = bench.dominant_roofline("dslash_df", tc, nc, w, {"hbm_gbs": 6000.0}, 2070.0)
    flops = 1320.0 * V * 2 * w["n_rhs"]                   # two-sided: A and A^dagger
    assert r["flops_per_launch"] == pytest.approx(flops)
    assert r["achieved"] == pytest.approx(flops / 1e-4 / 1e12)
    assert r["peak"] == pytest.approx(152 * 128 * 2070e6 / 9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])


def test_roofline_of_step2_averages_its_launches():
    """Launches j1 <= j <= k - 2; those before an FP32 stencil (j + 1 >= j0)
    also write the FP32 copies: 128 B per element two-sided, else 112 B."""
    w = dict(bench.WORKLOADS[bench.DEFAULT_WORKLOAD], k=10, j0=4, j1=0)
    V = int(np.prod(w["dims"]))
    N = 12 * V
    n = 9                                  # j = 0 .. 8
    n_copy = 6                             # j = 3 .. 8
    tc, nc = {"step2_df": 0.09}, {"step2_df": n}   # 10 us per launch
    r = bench.dominant_roofline("step2_df", tc, nc, w, {"hbm_gbs": 6000.0}, 2070.0)
    per_el = (n_copy * 128 + (n - n_copy) * 112) / n
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(per_el * N * w["n_rhs"])
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)


def test_committed_profiles_give_the_traffic_of_the_outer_kernels():
    for k in ("k_dslash_step1<df>", "k_dslash_step1<float>", "k_step2_df"):
        t = bench.profiled_traffic(k)
        assert t is not None and 1e7 < t < 1e9, k
    assert bench.profiled_traffic("no_such_kernel") is None


def test_config_names_the_workload_and_its_schedule():
    w = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    c = bench.config_of(w, _args())
    assert c["workload"] == bench.DEFAULT_WORKLOAD
    assert c["lattice"] == "x".join(str(d) for d in w["dims"])
    assert c["batches_in_flight"] == 4
    assert c["k"] == w["k"] and c["ell"] == w["ell"] and c["n_rhs"] == w["n_rhs"]
    assert ("before step %d" % bench.j1_of(w, _args())) in c["precision"]
