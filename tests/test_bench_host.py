"""Host helpers of bench.py that decide what the JSON line reports: the tensor
peak per operand format, the measured-peaks file, the DRAM traffic taken from
the committed profile only while the kernel source is unchanged, and the
clock samples kept for the timed region."""
import os
import subprocess
import time
from datetime import datetime

import pytest

import bench


def test_gemm_peak_ratios():
    """Burst figure by default (the GEMM is timed in a short region), sustained
    on request; TF32 / E4M3 take their own measured figures when recorded, else
    the BF16 figure times the nominal ratio; 3xTF32 is a third of TF32."""
    peaks = {"bf16_tflops": 1500.0, "bf16_tflops_sustained": 1200.0}
    pk = lambda c, **kw: bench.gemm_peak_tflops(c, peaks, **kw)[0]  # noqa: E731
    assert pk("bf16") == 1500.0 and pk("f16") == 1500.0
    assert pk("bf16", burst=False) == 1200.0
    assert pk("tf32") == 750.0 and pk("tf32", burst=False) == 600.0
    assert pk("f32") == pytest.approx(250.0)  # 3 TF32 products
    assert pk("e4m3") == 3000.0
    meas = {"tf32_tflops": 900.0, "e4m3_tflops": 2800.0, "e4m3_tflops_sustained": 2500.0}
    assert pk("tf32", measured=meas) == 900.0
    assert pk("f32", measured=meas) == pytest.approx(300.0)
    assert pk("e4m3", measured=meas) == 2800.0
    assert pk("e4m3", burst=False, measured=meas) == 2500.0
    assert pk("tf32", burst=False, measured=meas) == 600.0  # no sustained TF32 recorded
    assert "measured e4m3_tflops" in bench.gemm_peak_tflops("e4m3", peaks, measured=meas)[1]


def test_tensor_peaks_profile(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.tensor_peaks() == {}
    (prof / bench.TENSOR_PEAKS_PROFILE).write_text(
        "# notes\ntf32_tflops: 950.5\ne4m3_tflops: 3.1e3\ne4m3_tflops_sustained: 2700\n")
    assert bench.tensor_peaks() == {"tf32_tflops": 950.5, "e4m3_tflops": 3100.0,
                                    "e4m3_tflops_sustained": 2700.0}


def test_measured_peaks_file_or_fallback(tmp_path, monkeypatch):
    peaks, src = bench.measured_peaks()
    assert src in ("measured", "fallback")
    assert peaks["bf16_tflops_sustained"] > 0 and peaks["hbm_gbs"] > 0
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.measured_peaks()
    assert src == "fallback" and peaks == {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                                           "bf16_tflops_sustained": 1700.0}


def test_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    sha = bench.gemm_source_sha()
    prof = tmp_path / "profiles"
    prof.mkdir()
    src = tmp_path / "paper_1511_05690_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in ("pn_gemm_kernel.cuh", "pn_device.cuh", "pn_internal.h"):
        (src / f).write_bytes(open(os.path.join(bench.ROOT, "paper_1511_05690_gb300", "csrc",
                                                f), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.gemm_source_sha() == sha
    (prof / "gemm_level_bf16_n16384.md").write_text(
        f"kernel_source_sha256_16: {sha}\ntraffic_bytes_per_launch: 1.25e9\n")
    assert bench.traffic_from_profile("bf16") == 1.25e9
    (prof / "gemm_level_bf16_n16384.md").write_text(
        "kernel_source_sha256_16: 0123456789abcdef\ntraffic_bytes_per_launch: 1.25e9\n")
    assert bench.traffic_from_profile("bf16") is None  # kernel changed since the capture
    assert bench.traffic_from_profile("e4m3") is None  # no profile for this format


def _sampler_with(tmp_path, rows, t0, t1):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        for ts, sm, mx, reasons in rows:
            stamp = datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
            f.write(f"{stamp}, 0, {sm}, {mx}, 900.0, 0x0, " + ", ".join(reasons) + "\n")
        f.write("garbage line\n")
    s.proc = subprocess.Popen(["sleep", "30"])
    s.t0, s.t1 = t0, t1
    return s


def test_clock_samples_inside_the_timed_region(tmp_path):
    now = time.time()
    na = ["Not Active"] * 4
    cap = ["Not Active", "Not Active", "Not Active", "Active"]
    rows = [(now - 5, 1000, 2070, ["Active"] * 4),      # before the region: ignored
            (now + 0.1, 2070, 2070, na), (now + 0.2, 1950, 2070, cap),
            (now + 0.3, 2070, 2070, na), (now + 9, 800, 2070, ["Active"] * 4)]
    out = _sampler_with(tmp_path, rows, now, now + 1.0).stop()
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert out["sampling"] == "inside timed region"


def test_clock_nearest_sample_for_a_short_region(tmp_path):
    now = time.time()
    rows = [(now - 1.0, 1500, 2070, ["Not Active"] * 4),
            (now + 0.06, 2010, 2070, ["Active", "Not Active", "Not Active", "Not Active"])]
    out = _sampler_with(tmp_path, rows, now + 0.04, now + 0.05).stop()
    assert out["sm_mhz"] == 2010 and out["samples"] == 1
    assert out["reasons"] == ["hw_slowdown"] and out["sampling"].startswith("nearest")
