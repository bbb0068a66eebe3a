"""CPU-only checks of bench.py's host arithmetic: the algorithmic bytes per
cell-step of each configuration, the roofline fields, the recorded DRAM
traffic (used only while the kernel sources match the capture), the clock
sampler's reading of nvidia-smi rows, the accuracy record and the whole-job
rate of one rank."""
import json
import os

import numpy as np
import pytest

import bench


def test_algorithmic_bytes_per_cell_step():
    # (8 nvar + 1) w: 2-D gas FP32 / FP64, 3-D gas FP32, elastoplastic impact FP32
    assert bench.bytes_per_cell_step(5, 4) == 164
    assert bench.bytes_per_cell_step(5, 8) == 328
    assert bench.bytes_per_cell_step(6, 4) == 196
    assert bench.bytes_per_cell_step(12, 4) == 388


def test_roofline_fields():
    r = bench.roofline(4.0e9, 2.0, 6800.0, "measured", "k")
    assert r["achieved"] == pytest.approx(2000.0)
    assert r["frac"] == pytest.approx(2000.0 / 6800.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["avg_launch_ms"] == 2.0
    assert bench.roofline(1.0, 1.0, 1.0, "measured", "k", {"traffic": 5})["traffic"] == 5


def test_recorded_traffic_is_consistent_and_tied_to_the_sources(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "batch_step_ellipses_fp32.json")) as f:
        d = json.load(f)
    assert d["dram_bytes_per_cell_step"] == pytest.approx(d["dram_bytes_per_step"] / d["cells"], abs=0.01)
    assert d["dram_bytes_per_cell_step"] < d["algorithmic_bytes_per_cell_step"] == 164
    monkeypatch.setattr(bench, "kernel_hash", lambda: d["kernel_source_hash"])
    assert bench.recorded_traffic("batch_step_ellipses_fp32.json")["dram_bytes_per_step"] == d["dram_bytes_per_step"]
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("batch_step_ellipses_fp32.json") is None
    assert bench.recorded_traffic("no_such_record.json") is None


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def sampled(tmp_path, lines):
    c = bench.Clocks.__new__(bench.Clocks)
    c.f = open(tmp_path / "clocks.csv", "w+")
    c.f.write("\n".join(lines) + "\n")
    c.p = _Done()
    return c.stop()


def test_clock_sampler_reads_median_and_reasons(tmp_path):
    row = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {pc}"
    out = sampled(tmp_path, [row.format(sm=2070, hw="Not Active", pc="Not Active"),
                             row.format(sm=1980, hw="Not Active", pc="Active"),
                             row.format(sm=2070, hw="Not Active", pc="Not Active"),
                             "garbage line"])
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    out = sampled(tmp_path, [row.format(sm=1500, hw="Active", pc="Not Active")])
    assert out["reasons"] == ["hw_slowdown"] and out["sm_mhz"] == 1500.0


def test_accuracy_record_measures_l1_and_front_offset():
    spec = ("cylinder", (64,))
    wl = bench.make_workload(spec)
    ref = np.zeros((5, wl.ncell))
    ref[0] = 1.0
    ref[3] = 2.5e5
    row = bench.shock_row(spec, wl)
    j, _ = row
    line = np.ones(64)
    line[:20] = 3.0                              # a front between cells 19 and 20
    ref[0].reshape(-1, 64)[j] = line
    front = bench.front_index(bench.density_line(ref, wl), wl, row)
    assert front == 19
    same = bench.accuracy_record(ref.copy(), ref, wl, spec, front, 10)
    assert same["rel_l1_max"] == 0.0 and same["front_offset_cells"] == 0
    got = ref.copy()
    shifted = np.ones(64)
    shifted[:21] = 3.0
    got[0].reshape(-1, 64)[j] = shifted
    rec = bench.accuracy_record(got, ref, wl, spec, front, 10)
    assert rec["front_cell_gpu"] == 20 and rec["front_offset_cells"] == 1
    assert rec["rel_l1_per_plane"][0] == pytest.approx(2.0 / np.abs(ref[0]).sum())
    assert rec["rel_l1_per_plane"][3] == 0.0


def test_whole_job_rate_of_one_rank():
    rate, slowest = bench.whole_job_rate(2.0, 1000, 1, "cpu")
    assert slowest == 2.0 and rate == pytest.approx(1000 / 2e-3)
