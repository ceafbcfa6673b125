"""Host logic of bench.py (no GPU): when a committed DRAM-traffic figure may be reported, and how
the clock sampler reads nvidia-smi's throttle reasons."""
import os
import shutil
import subprocess

import pytest

import bench

CSRC = os.path.join(bench.ROOT, "paper_2402_00525_gb300", "csrc")


def test_traffic_is_reported_only_for_the_captured_sources_and_workload(monkeypatch):
    fwd = bench.measured_traffic("k_render<4,0>", 3_000_000, 16)
    bwd = bench.measured_traffic("k_render_bwd_list", 3_000_000, 16)
    # the committed capture matches the Render sources of this checkout
    assert fwd is not None and bwd is not None and fwd > bwd > 1e9
    # another workload size: the capture does not describe it
    assert bench.measured_traffic("k_render<4,0>", 500_000, 16) is None
    assert bench.measured_traffic("k_render<4,0>", 3_000_000, 8) is None
    # changed Render code: the figure is stale and is not reported
    monkeypatch.setattr(bench, "render_source_hash", lambda: "0" * 64)
    assert bench.measured_traffic("k_render<4,0>", 3_000_000, 16) is None


def test_source_hash_follows_code_not_comments(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    dst = root / "paper_2402_00525_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.RENDER_SOURCES:
        shutil.copy(os.path.join(CSRC, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    h0 = bench.render_source_hash()
    assert h0 == bench.render_source_hash()
    path = dst / "stp_render.cu"
    txt = path.read_text()
    path.write_text("// a new comment line\n/* and a block\n comment */\n" + txt.replace("\n", "\n  ", 3))
    assert bench.render_source_hash() == h0                 # comments and whitespace only
    path.write_text(txt.replace("kFifo", "kFifoRenamed", 1))
    assert bench.render_source_hash() != h0                 # a code change


class _FakeSmi:
    """Stands in for `nvidia-smi --query-gpu ... -lms 200`: writes canned rows to its stdout."""
    rows = []

    def __init__(self, cmd, stdout=None, stderr=None):
        assert cmd[0] == "nvidia-smi" and any(a.startswith("--query-gpu=") for a in cmd)
        stdout.write("".join(r + "\n" for r in self.rows))
        stdout.flush()

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def test_clock_sampler_reads_median_clock_and_throttle_reasons(monkeypatch):
    _FakeSmi.rows = [
        "0, 2070 MHz, 2070 MHz, 900.00 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055 MHz, 2070 MHz, 1390.00 W, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070 MHz, 2070 MHz, 1200.00 W, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbled line",
    ]
    monkeypatch.setattr(subprocess, "Popen", _FakeSmi)
    cs = bench.ClockSampler(0)
    cs.start()
    got = cs.stop()
    assert got["sm_mhz"] == 2070.0 and got["sm_max_mhz"] == 2070.0 and got["samples"] == 3
    assert got["reasons"] == ["sw_power_cap"]               # kept and noted, not a rejection
    _FakeSmi.rows = [
        "0, 1400 MHz, 2070 MHz, 800.00 W, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "0, 1410 MHz, 2070 MHz, 800.00 W, 0x0000000000000020, Not Active, Active, Not Active, Not Active",
    ]
    cs = bench.ClockSampler(0)
    cs.start()
    got = cs.stop()
    assert got["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]      # a run to re-measure
    assert got["sm_mhz"] == pytest.approx(1405.0)


def test_clock_sampler_without_nvidia_smi(monkeypatch):
    def missing(*a, **k):
        raise FileNotFoundError("nvidia-smi")
    monkeypatch.setattr(subprocess, "Popen", missing)
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
