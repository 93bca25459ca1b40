"""Host logic of bench.py that decides what the JSON line reports: the
timing method of the timed region and the measured-traffic lookup. No GPU
is involved (fake events)."""
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


def test_measured_traffic_follows_the_kernel_source(monkeypatch, tmp_path):
    # a traffic record of 600 MB per 8-step launch of a 2000 x 12500 grid,
    # keyed by a kernel source hash
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "blocked_stencil_traffic.json").write_text(json.dumps({
        "kernel_src_sha": "abc", "block_steps": 8, "cells": 25_000_000,
        "dram_bytes_per_launch": 600_000_000}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    spec = types.SimpleNamespace(nx=2000, ny=12500)
    assert bench.measured_traffic(spec, 8) == 600_000_000
    half = bench.measured_traffic(types.SimpleNamespace(nx=1000, ny=12500), 8)
    assert half == 300_000_000                                  # scaled by cells
    assert bench.measured_traffic(spec, 7) is None              # another depth
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "def")
    assert bench.measured_traffic(spec, 8) is None              # changed kernel
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "missing"))
    assert bench.measured_traffic(spec, 8) is None              # no record
