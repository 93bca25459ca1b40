"""Host logic of bench.py that decides what the JSON line reports: the
timing method of the timed region, the lookup of the ncu counter record, the
issue and DRAM fractions and the R/T check against stored oracle runs. No
GPU is involved (fake events and device properties)."""
import json
import types

import bench


class _Ev:
    def __init__(self, ms=None, fail=False):
        self.ms, self.fail = ms, fail

    def elapsed_time(self, other):
        if self.fail:
            raise RuntimeError("event not recorded")
        return other.ms - self.ms


def test_events_are_used_when_they_span_the_work():
    t, how = bench.event_seconds(_Ev(0.0), _Ev(980.0), wall=1.0)
    assert t == 0.98 and how.startswith("CUDA events")


def test_wall_clock_when_events_fail_or_miss_the_work():
    t, how = bench.event_seconds(_Ev(fail=True), _Ev(5.0), wall=1.25)
    assert t == 1.25 and "wall clock" in how
    # events on a stream that did not carry the work span almost nothing
    t, how = bench.event_seconds(_Ev(0.0), _Ev(3.0), wall=1.25)
    assert t == 1.25 and "wall clock" in how


def test_measured_counters_follow_kernel_shape_and_plan(monkeypatch, tmp_path):
    # a counter record of one 8-step launch of a 2000 x 12500 grid, keyed by
    # the kernel source, the depth, the code shape and the segment plan
    (tmp_path / "profiles").mkdir()
    rec = {"kernel_src_sha": "abc", "block_steps": 8, "variant": 5, "plan_sha": "p1",
           "cells": 25_000_000, "dram_bytes_per_launch": 600_000_000,
           "warp_inst_per_launch": 80_000_000}
    (tmp_path / "profiles" / "blocked_stencil_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    spec = types.SimpleNamespace(nx=2000, ny=12500)
    d = bench.measured_counters(spec, 8, 5, "p1")
    assert d["dram_bytes_per_launch"] == 600_000_000 and d["warp_inst_per_launch"] == 80_000_000
    assert bench.measured_counters(spec, 7, 5, "p1") is None          # another depth
    assert bench.measured_counters(spec, 8, 2, "p1") is None          # another code shape
    assert bench.measured_counters(spec, 8, 5, "p2") is None          # another plan
    other = types.SimpleNamespace(nx=1000, ny=12500)
    assert bench.measured_counters(other, 8, 5, "p1") is None         # another grid
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "def")
    assert bench.measured_counters(spec, 8, 5, "p1") is None          # changed kernel
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "missing"))
    assert bench.measured_counters(spec, 8, 5, "p1") is None          # no record


def test_golden_rt_check_compares_matching_runs(monkeypatch, tmp_path):
    g = tmp_path / "tests" / "golden"
    g.mkdir(parents=True)
    (g / "oracle_c2_550nm.json").write_text(
        json.dumps({"steps": 30000, "R": 0.1, "T": 0.5, "polarization": "S (TMz)"}))
    (g / "oracle_c2_800nm.json").write_text(
        json.dumps({"steps": 4000, "R": 0.2, "T": 0.4, "polarization": "S (TMz)"}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    res = [(550e-9, (0.1004, 0.4999)), (800e-9, (0.3, 0.3)), (450e-9, (0.0, 0.0))]
    d = bench.golden_rt_check(res, 30000, "s")
    # only the 550 nm run has a stored oracle run of the same length
    assert d["runs_checked"] == 1 and d["wavelengths_nm"] == [550]
    assert abs(d["max_abs_err_R"] - 4e-4) < 1e-12 and abs(d["max_abs_err_T"] - 1e-4) < 1e-12
    assert bench.golden_rt_check(res, 1000, "s") is None
    # the stored runs are S-polarised: a P line has nothing to compare with
    assert bench.golden_rt_check(res, 30000, "p") is None
    (g / "oracle_c2p_550nm.json").write_text(
        json.dumps({"steps": 30000, "R": 0.2, "T": 0.4, "polarization": "P (TEz)"}))
    d = bench.golden_rt_check(res, 30000, "p")
    assert d["runs_checked"] == 1 and abs(d["max_abs_err_R"] - 0.0996) < 1e-12


def test_issue_fraction_of_the_roofline_record(monkeypatch):
    import torch
    props = types.SimpleNamespace(multi_processor_count=152)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda i: props)
    r = bench.roofline_record(35000.0, 6785.2, "measured", 5e9, 1.4e-4, 6.25e8, 1.1e8,
                              {"sm_mhz": 2070.0})
    assert r["bound"] == "issue" and abs(r["frac"] - 35000.0 / 6785.2) < 1e-12
    peak = 152 * 4 * 2070e6
    assert abs(r["issue_frac"] - 1.1e8 / 1.4e-4 / peak) < 1e-12
    assert abs(r["dram_frac"] - 6.25e8 / 1.4e-4 / 1e9 / 6785.2) < 1e-12
    r = bench.roofline_record(35000.0, 6785.2, "measured", 5e9, 1.4e-4, None, None, None)
    assert r["issue_frac"] is None and r["dram_frac"] is None and r["traffic"] is None
