"""The bench's clock record from a fake NVML (no GPU, no driver library): the median SM clock,
the maximum, and the union of the clock-event reasons seen while sampling."""
import importlib.util
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.path.insert(0, ROOT)
    spec.loader.exec_module(mod)
    return mod


class _FakeNvml:
    def __init__(self, seq):
        self.seq = list(seq)
        self.i = 0
        self.closed = False

    def sample(self):
        v = self.seq[min(self.i, len(self.seq) - 1)]
        self.i += 1
        return v

    def close(self):
        self.closed = True


def test_clock_summary_from_fake_nvml(monkeypatch):
    bench = _bench()
    seq = [(1900.0, 2070.0, set()), (2070.0, 2070.0, {"sw_power_cap"}), (2070.0, 2070.0, set())]
    fake = _FakeNvml(seq)
    monkeypatch.setattr(bench, "_NvmlClocks", lambda idx: fake)
    cs = bench.ClockSampler(0)
    cs.start()
    time.sleep(0.05)
    out = cs.stop()
    assert fake.closed
    assert out["samples"] >= 3
    assert out["sm_max_mhz"] == 2070.0
    assert out["sm_mhz"] == 2070.0          # the median of the samples
    assert out["reasons"] == ["sw_power_cap"]
    assert "NVML" in out["source"]


def test_clock_reason_bits():
    bench = _bench()
    bits = bench._NvmlClocks.BITS
    # the reasons that reject a run must all be decoded
    assert set(bits.values()) >= {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"}
    assert len(set(bits)) == len(bits) and all(b & (b - 1) == 0 for b in bits)


def test_no_nvml_no_smi_gives_none(monkeypatch):
    bench = _bench()

    def boom(idx):
        raise OSError("no NVML")
    monkeypatch.setattr(bench, "_NvmlClocks", boom)
    monkeypatch.setenv("PATH", "/nonexistent")
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop() is None


def test_clock_summary_from_fake_nvidia_smi(monkeypatch, tmp_path):
    """Without NVML the sampler reads nvidia-smi's CSV (a fake on PATH here): median and maximum
    SM clock, and every throttle reason reported Active."""
    bench = _bench()

    def boom(idx):
        raise OSError("no NVML")
    monkeypatch.setattr(bench, "_NvmlClocks", boom)
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "echo '0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "echo '0, 1950, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "echo '0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "exec sleep 30\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ.get('PATH', '')}")
    cs = bench.ClockSampler(0)
    cs.start()
    time.sleep(0.5)
    out = cs.stop()
    assert out is not None
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert "nvidia-smi" in out["source"]
