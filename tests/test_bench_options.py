"""The benchmark's host logic on CPU: option plumbing into the workload
description, the two-dimensional cell parser, the cpulist parser of the e2e
leg's host-buffer placement, the traffic lookup's shape check and the oracle
arm's JSON line with method options."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_grid_cells_parse():
    assert bench.grid_cells(None) is None
    assert bench.grid_cells("4x16") == (4, 16)
    assert bench.grid_cells("1X32") == (1, 32)


def test_cpulist_parse_and_no_gpu_means_no_affinity_change():
    assert bench.parse_cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench.parse_cpulist("5") == {5}
    assert bench.parse_cpulist("") == set()
    # without a GPU (or its sysfs entry) the e2e leg leaves the affinity alone
    import torch
    if not torch.cuda.is_available():
        assert bench.gpu_local_cpus(0) == set()


def test_workload_config_names_every_option():
    c = bench.workload_config(48)
    assert "768 units x 256 ch x 3072 t" in c["workload"]
    assert not {"sir_percent", "time_mode", "stats_scope", "sigma_estimator"} & set(c)
    c = bench.workload_config(4, sir=20, scope=True, sigma="winsor")
    assert c["sir_percent"] == 20 and c["stats_scope"] == "per channel"
    assert c["sigma_estimator"] == "winsor" and c["per_rank_units"] == 64
    assert "integrated" in bench.workload_config(48, integrated=True)["time_mode"]
    assert "4 x 16" in bench.workload_config(48, grid="4x16")["time_mode"]


def test_traffic_only_for_the_profiled_shape():
    default = dict(threads=256, ctas_per_sm=2, tile_bytes=0, fine_bins=2048, flag_rows=64,
                   stat_samples=262144)
    t = bench.measured_traffic(768, default)
    other = bench.measured_traffic(768, dict(default, flag_rows=32))
    assert other is None
    if t is not None:                     # the kernel sources still match the recorded hashes
        assert t == 768 * bench.measured_traffic(1, default)


def test_roofline_entry():
    r = bench.roofline_entry(5.4358e9, 4.4, 6775.3, "measured", 7.0e9, "lof_block_kernel<CI16>")
    assert r["achieved"] == pytest.approx(5.4358e9 / 4.4e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6775.3)
    assert r["frac_nominal"] == pytest.approx(r["achieved"] / 7900.0)
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(r)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 7.0e9


def test_timed_kernel_names():
    import argparse
    a = argparse.Namespace(grid=None, integrated=False, channel_scope=False, sigma="mad", sir=0)
    assert bench.timed_kernel_name(a) == "lof_block_kernel<CI16>"
    assert bench.timed_kernel_name(argparse.Namespace(**dict(vars(a), sir=20))).endswith("+ SIR")
    assert "two-dimensional" in bench.timed_kernel_name(argparse.Namespace(**dict(vars(a), grid="4x16")))
    assert "pooled exact" in bench.timed_kernel_name(argparse.Namespace(**dict(vars(a), sigma="winsor")))


def test_reference_arm_with_options():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.5",
                          "--grid", "4x16", "--sigma", "winsor"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["sigma_estimator"] == "winsor"
    assert "4 x 16" in line["config"]["time_mode"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]


def test_gpu_line_assembly_with_a_fake_run(monkeypatch, capsys):
    # main()'s JSON line from a stand-in for run_gpu's timings: every key of
    # the contract present, the roofline built from the kernel time
    res = {"rank": 0, "value": 133000.0, "ms_per_step": 4.5, "step_ms": [4.5, 4.6, 4.4],
           "kern_ms": [4.4, 4.4, 4.4], "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []},
           "samples": 768 * 256 * 3072, "plain_ms": [120.0, 119.0, 121.0],
           "tuning": dict(threads=256, ctas_per_sm=2, tile_bytes=0, fine_bins=2048, flag_rows=64,
                          stat_samples=262144),
           "e2e": {"value": 16000.0, "unit": "Msamples/s", "h2d_bytes_per_step": 1,
                   "d2h_bytes_per_step": 1},
           "refine": [{"units_refined": 0, "refine_passes": 0}, {"units_refined": 2, "refine_passes": 6}]}
    monkeypatch.setattr(bench, "run_gpu", lambda args: res)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    for extra, kernel in (([], "lof_block_kernel<CI16>"), (["--grid", "4x16"], "two-dimensional")):
        monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", "3", "--warmup", "3", "--no-cpu"] + extra)
        bench.main()
        line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
        for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                  "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "e2e",
                  "gpu_launches", "latency_ms"):
            assert k in line, k
        r = line["roofline"]
        assert r["kernel_ms"] == pytest.approx(4.4) and kernel in r["kernel"]
        assert r["achieved"] == pytest.approx(res["samples"] * 9 / 4.4e-3 / 1e9)
        assert line["gpu_launches"] == 2 * 3
        assert line["plain_vs_batched"] == pytest.approx(120.0 / 4.4)
        assert line["stats_refinement"]["units_refined_per_launch"] == [0, 2]
        if not extra:
            assert r["traffic"] == bench.measured_traffic(768, res["tuning"])
        else:
            assert r["traffic"] is None
