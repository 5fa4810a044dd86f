"""Host logic of bench.py on the CPU: the clock sampler (against a stand-in
nvidia-smi that prints the queried fields), the launch count of one step and
the DRAM traffic taken from an ncu summary only while the kernel's source is
the one profiled."""
import hashlib
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth_inputs as S  # noqa: E402


def _fake_smi(tmp_path, line, delay=0.2):
    p = tmp_path / "nvidia-smi"
    p.write_text(f"#!/bin/sh\nsleep {delay}\nwhile true; do echo '{line}'; sleep 0.05; done\n")
    p.chmod(p.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def test_clock_sampler_reads_clocks_and_reasons(tmp_path, monkeypatch):
    d = _fake_smi(tmp_path, "1980, 2070, 1350.5, 0x4, Not Active, Not Active, Not Active, Active")
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    t0 = time.perf_counter()
    c.start()
    assert time.perf_counter() - t0 < 3.5        # waited for the first sample, bounded
    time.sleep(0.4)
    r = c.stop()
    assert r["samples"] >= 2
    assert r["sm_mhz"] == 1980.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_sampler_keeps_only_samples_after_start(tmp_path, monkeypatch):
    # stopped at once: the sample that announced the process is not counted
    d = _fake_smi(tmp_path, "2070, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, Not Active", 0.0)
    monkeypatch.setenv("PATH", d + os.pathsep + os.environ["PATH"])
    c = bench.ClockSampler(0)
    c.start()
    r = c.stop()
    assert r["samples"] <= 1


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_launches_per_step():
    wl = S.WORKLOADS["zoom2x_512_dict1m"]
    # features, hash, lookup; 9 launches of the three-stage search; LLE, the
    # two overlap-average passes; 2 per back-projection step
    assert bench.launches_per_step(wl, True) == 3 + 9 + 3 + 2 * wl.bp_iters == 25
    assert bench.launches_per_step(wl, False) == 17


def test_profiled_traffic_follows_the_source(tmp_path):
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    summ = tmp_path / "s.md"
    summ.write_text(f"# capture\n\nCommand: ncu ...\n\nkernel_source_sha256_16: {sha}\n"
                    "traffic_bytes_per_launch: 123456\n")
    assert bench.profiled_traffic(str(src), str(summ)) == 123456
    src.write_text("__global__ void k() { }\n")          # the kernel changed: no traffic
    assert bench.profiled_traffic(str(src), str(summ)) is None
    assert bench.profiled_traffic(str(src), str(tmp_path / "missing.md")) is None

