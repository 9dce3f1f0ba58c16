"""Host-side logic of bench.py that needs no GPU: the clock/throttle summary taken from
nvidia-smi samples (fed here from a fake sampler, as nvidia-smi would print them) and the
DRAM-traffic figure read from the committed ncu summary only while it matches the
kernel source."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _FakeThread:
    def join(self, timeout=None):
        pass


def _sampler(lines):
    s = bench.ClockSampler()
    s.proc, s.thread, s.lines = _FakeProc(), _FakeThread(), list(lines)
    return s


def _row(sm, smax=2070, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    # the columns of ClockSampler.FIELDS, csv,noheader,nounits
    return f"{sm}, {smax}, 850.31, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_max_and_no_reason():
    out = _sampler([_row(2070), _row(2070), _row(1980), "garbage line"]).stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == [] and out["samples"] == 3


@pytest.mark.parametrize("field,name", [("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                                        ("swt", "sw_thermal_slowdown"), ("cap", "sw_power_cap")])
def test_clock_summary_reports_each_throttle_reason(field, name):
    out = _sampler([_row(2070), _row(1500, **{field: "Active"})]).stop()
    assert out["reasons"] == [name]


def test_clock_summary_without_samples():
    assert _sampler(["[N/A], [N/A]"]).stop()["reasons"] == ["no samples"]
    s = bench.ClockSampler()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_profiled_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    prof = tmp_path / "k_step.md"
    prof.write_text("kernel_source_sha256_16: 0123456789abcdef\ndram_bytes_per_launch_full_size: 3.5e9\n")
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0123456789abcdef")
    assert bench.profiled_traffic() == 3.5e9
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "fedcba9876543210")
    assert bench.profiled_traffic() is None
    monkeypatch.setattr(bench, "PROFILE", str(tmp_path / "missing.md"))
    assert bench.profiled_traffic() is None


def test_committed_profile_names_a_hash_and_a_traffic_figure():
    txt = open(bench.PROFILE).read()
    assert "kernel_source_sha256_16:" in txt and "dram_bytes_per_launch_full_size:" in txt
