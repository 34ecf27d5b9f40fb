"""Host logic of bench.py on the CPU: the clock record, the ncu traffic read
from a committed profile, the roofline arithmetic (algorithmic bytes counted
by hand on a small probe pattern), and the reference arm's JSON line, which
runs the oracle alone and so needs no GPU."""
import json
import os
import subprocess
import sys
import types

import pytest
import torch

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _clock_line(sm, mx, hw="Not Active", hw_th="Not Active", sw_th="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.0, 0x0, {hw}, {hw_th}, {sw_th}, {cap}"


def test_clock_summary_takes_the_median_and_collects_reasons():
    s = bench.ClockSampler(0)
    s.lines = [_clock_line(2070, 2070), _clock_line(1980, 2070, cap="Active"), _clock_line(2040, 2070),
               "garbage", _clock_line("[N/A]", 2070)]
    out = s.summary()
    assert out["sm_mhz"] == 2040 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    s.lines = [_clock_line(1500, 2070, hw="Active", hw_th="Active", sw_th="Active")]
    assert s.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    s.lines = []
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}


def test_committed_scan_profile_was_taken_on_the_current_kernel_source():
    # roofline.traffic comes from this summary only while its source hash
    # matches the scan kernel's sources; a kernel change without a new
    # capture makes it null
    path = os.path.join(ROOT, "profiles", f"{bench.SCAN_KERNEL}_glove.txt")
    txt = open(path).read()
    assert f"source_hash: {bench.kernel_hash()}" in txt
    traffic = bench.profiled_traffic("glove")
    assert traffic is not None and 0.9e9 < traffic < 1.3e9


def test_profiled_traffic_is_null_for_another_source_or_workload(monkeypatch):
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0000000000000000")
    assert bench.profiled_traffic("glove") is None
    assert bench.profiled_traffic("no_such_workload") is None


class _FakeBinding:
    def __init__(self, top):
        self.top = top

    def soar_select_partitions(self, ix, Qd, t):
        assert self.top.shape[1] == t
        return self.top


class _FakeIndex:
    def __init__(self, offsets):
        self._off = torch.tensor(offsets, dtype=torch.int64)

    def offsets(self):
        return self._off


def test_scan_roofline_counts_each_probed_partition_once():
    # 4 partitions of 10, 20, 0 and 15 rows; 3 queries probing 2 each
    w = types.SimpleNamespace(c=4, d=8)
    top = torch.tensor([[0, 1], [1, 3], [0, 1]], dtype=torch.int32)
    ix = _FakeIndex([0, 10, 30, 30, 45])
    k, nq, t, ms = 10, 3, 2, 1e-3
    r = bench.scan_roofline(w, nq, k, t, ix, None, _FakeBinding(top), ms, 6785.2, 1916.2, "measured")
    rows_once = 10 + 20 + 15                          # partitions 0, 1, 3, each once
    want = rows_once * (4 * 8 + 4) + nq * 4 * 8 + nq * k * 12
    assert r["algorithmic_bytes"] == want
    assert r["achieved"] == pytest.approx(want / (ms / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6785.2)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == 6785.2
    assert r["schedule_bytes"]["rows_rereads"] == 0  # no partition has more than 128 queries
    assert r["algorithmic_flops"] == 2 * 8 * (10 + 20 + 20 + 15 + 10 + 20)


def test_scan_roofline_reports_rereads_of_partitions_beyond_128_queries():
    # 130 queries probe partition 0 (two 128-query chunks): its rows are read
    # twice by the kernel's schedule, once by the algorithmic count
    w = types.SimpleNamespace(c=2, d=100)
    top = torch.zeros((130, 1), dtype=torch.int32)
    ix = _FakeIndex([0, 64, 100])
    r = bench.scan_roofline(w, 130, 1, 1, ix, None, _FakeBinding(top), 1.0, 6785.2, 1916.2, "measured")
    assert r["algorithmic_bytes"] == 64 * (4 * 100 + 4) + 130 * 400 + 130 * 12
    assert r["schedule_bytes"]["rows_rereads"] == 64 * 104 * 4     # d padded to 104
    assert r["schedule_bytes"]["candidate_list_capacity"] == 130 * 1 * 8 * 128


def test_assign_roofline_counts_primary_and_spill_passes():
    w = types.SimpleNamespace(n=1000, c=50, d=100)
    r = bench.assign_roofline(w, 2.0, 1916.2, "measured")
    assert r["tf32_tflops"] == pytest.approx(6 * 1000 * 50 * 100 / 2e-3 / 1e12)
    assert r["tf32_peak_tflops"] == pytest.approx(958.1)
    assert r["assignments_per_s"] == pytest.approx(1000 / 2e-3)
    assert r["alu_pairs_peak_per_s"] == pytest.approx(152 * 128 * 2070e6 / 8)


def test_peaks_are_the_measured_ones_else_the_fallback(monkeypatch, tmp_path):
    hbm, bf16, src = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        m = json.load(open(path))
        assert (hbm, bf16, src) == (m["hbm_gbs"], m["bf16_tflops"], "measured")
    else:
        assert (hbm, bf16, src) == (bench.FALLBACK_HBM_GBS, bench.FALLBACK_BF16_TFLOPS, "fallback")
    monkeypatch.setattr(bench, "MEASURED_PEAKS", str(tmp_path / "absent.json"))
    assert bench.peaks() == (6800.0, 1900.0, "fallback")


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
           "--cpu-sample", "32", "--steps", "2", "--warmup", "1"]
    return subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_contract_line_on_the_cpu():
    r = _run_reference({"RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["unit"] == "queries/s" and line["higher_is_better"] is True
    assert line["config"]["workload"].startswith("tiny")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "queries/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    r = _run_reference({"RANK": "1"})
    assert r.returncode == 0
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_time_oracle_reports_rate_wall_time_and_cpu_use():
    import synth
    w = synth.WORKLOADS["tiny"]
    X, Q, _ = synth.workload_arrays("tiny", n=4000, nq=40)
    C, off, ids = bench.oracle_index(X, w, w.lam, w.spills, train_rows=4000, iters=2)
    qps, secs, busy = bench.time_oracle(X, Q, C, off, ids, w.k, 4, 24)
    assert secs > 0 and qps == pytest.approx(24 / secs)
    assert busy > 0
    qps_all, _, _ = bench.time_oracle(X, Q, C, off, ids, w.k, 4, 10_000)   # more than there are
    assert qps_all > 0


def test_one_core_oracle_timing_runs_in_a_single_thread_child():
    import synth
    w = synth.WORKLOADS["tiny"]
    X, Q, _ = synth.workload_arrays("tiny", nq=40)
    C, off, ids = bench.oracle_index(X, w, w.lam, w.spills, train_rows=20_000, iters=2)
    rec = bench.time_oracle_one_core("tiny", Q, C, off, ids, w.k, 4, 32)
    assert "error" not in rec, rec
    assert rec["cores"] == 1 and rec["value"] > 0 and rec["kind"] == "oracle"
    assert rec["cpu_time_over_wall"] < 1.5                  # one thread did the work
    bad = bench.time_oracle_one_core("no_such_workload", Q, C, off, ids, w.k, 4, 8)
    assert set(bad) == {"error"} and "no_such_workload" in bad["error"]
