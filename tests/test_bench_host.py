"""Host-side pieces of bench.py that need no GPU: the clock record built
from nvidia-smi samples, the FP64 peak from unit counts and clock, the
measured-peak lookup and the traffic record's source check."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


class _FakeThread:
    def join(self, timeout=None):
        pass


def test_clock_record_from_samples():
    s = bench.ClockSampler(0)
    s.proc, s.thread = _FakeProc(), _FakeThread()
    s.lines = [
        "0, 1965, 2070, 850.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 910.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 905.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    rec = s.stop()
    assert rec == {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_record_absent_without_samples():
    s = bench.ClockSampler(0)
    assert s.stop() is None  # never started
    s.proc, s.thread, s.lines = _FakeProc(), _FakeThread(), []
    assert s.stop() is None


def test_fp64_peak_from_units_and_clock():
    assert bench.fp64_peak_tflops(2070.0) == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    assert bench.fp64_peak_tflops(None) == bench.fp64_peak_tflops(2070.0)


def test_measured_peak_lookup():
    value, kind = bench.measured_peak_gbs()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and value == float(json.load(open(path))["hbm_gbs"])
    else:
        assert (value, kind) == (6800.0, "fallback")


def test_traffic_record_only_for_its_sources():
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_faces_traffic.json.txt")))
    assert tuple(rec["sources"]) == bench.FACE_SOURCES
    got = bench.faces_traffic_from_profile()
    if rec["sources_sha1"] == bench.sources_sha1(bench.FACE_SOURCES):
        assert got == rec["dram_bytes_per_launch"]
    else:
        assert got is None
