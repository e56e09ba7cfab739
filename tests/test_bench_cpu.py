"""Host-side logic of the benchmark, on CPU: the DRAM traffic figure is taken
from the committed profile only while the profiled kernel source is
unchanged; the oracle timing helper steps every job it is given and counts
node updates correctly; the clock summary flags throttling."""
import hashlib
import os

import numpy as np

import bench


def test_traffic_is_read_only_for_the_profiled_kernel_source(tmp_path, monkeypatch):
    src = open(bench.KERNEL_SRC, "rb").read()
    digest = hashlib.sha256(src).hexdigest()[:16]
    prof = tmp_path / "prof.md"
    prof.write_text(f"- kernel_source_sha256_16: `{digest}`\n"
                    "- dram_bytes_per_launch_full_256: `123456789`\n")
    monkeypatch.setattr(bench, "PROFILE", str(prof))
    assert bench.profiled_traffic() == 123456789.0
    # any change to the kernel source voids the figure
    changed = tmp_path / "k.cu"
    changed.write_bytes(src + b"\n// changed\n")
    monkeypatch.setattr(bench, "KERNEL_SRC", str(changed))
    assert bench.profiled_traffic() is None


def test_committed_profile_matches_the_kernel_source():
    # the committed 3D profile is the one the bench line's traffic comes from
    assert bench.profiled_traffic() is not None


def test_oracle_jobs_rate_steps_every_job(oracle_lib):
    co = oracle_lib
    shapes = [(6, 8), (10, 12), (8, 8)]
    jobs, before = [], []
    for ny, nx in shapes:
        x = np.arange(nx) * 2 * np.pi / nx
        u = 0.01 * np.tile(np.sin(x), (ny, 1))
        f = [np.ones((ny, nx)), u, np.zeros((ny, nx)), None, None]
        jobs.append((co.make_params((ny, nx), nu=0.05), f))
        before.append(u.copy())
    rate, done, secs = bench.oracle_jobs_rate(jobs, 0.2, 2)
    assert rate > 0 and secs >= 0.2
    # every job moved, and the count is a whole number of steps of the jobs' sizes
    for (p, f), u0 in zip(jobs, before):
        assert not np.array_equal(f[1], u0)
    assert done % 2 == 0 and done >= sum(ny * nx for ny, nx in shapes)


def test_host_threads_is_positive():
    assert bench.host_threads() >= 1


def test_measured_peak_falls_back_without_the_file(monkeypatch, tmp_path):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, kind = bench.measured_peaks()
    assert kind == "fallback" and peak > 0
    if os.path.exists(os.path.join(os.path.dirname(bench.__file__), "MEASURED_PEAKS.json")):
        monkeypatch.undo()
        peak, kind = bench.measured_peaks()
        assert kind == "measured" and peak > 1000


def test_clock_summary_flags_throttle_reasons():
    c = bench.ClockSampler(0)
    # nvidia-smi --format=csv,noheader,nounits lines, as the sampler reads them
    c.lines = [
        "2070, 2070, 900.12, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, 1399.80, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1000.55, 0x0000000000000020, Not Active, Active, Not Active, Not Active",
        "garbage line",
    ]
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
