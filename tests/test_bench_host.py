"""CPU tests of bench.py's host logic: the clock-sample parser that decides
whether a run saw throttling, and the lookup of the screening kernel's DRAM
traffic in its committed ncu summary (only valid for the kernel source it was
taken on)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _write(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    return str(p)


def test_clock_parser_median_max_and_reasons(tmp_path):
    path = _write(tmp_path, [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2070, 1390.5, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
        "garbage line",                                                               # skipped
    ])
    r = bench.parse_clock_samples(path)
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_parser_reports_hardware_slowdown(tmp_path):
    path = _write(tmp_path, [
        "0, 1400, 2070, 1000, 0x8, Active, Not Active, Not Active, Not Active",
        "0, 1500, 2070, 1000, 0x8, Not Active, Active, Active, Not Active",
    ])
    r = bench.parse_clock_samples(path)
    assert r["sm_mhz"] == 1450.0 and r["samples"] == 2
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_parser_without_samples(tmp_path):
    assert bench.parse_clock_samples(_write(tmp_path, ["", "x,y"])) is None


def test_profile_traffic_only_for_the_profiled_source(monkeypatch):
    txt = open(os.path.join(ROOT, "profiles", "k_tc_screen_bf16_c2a.md")).read()
    per_row = float(txt.split("dram_bytes_per_row:")[1].split()[0])
    h = txt.split("source_sha256_16:")[1].split()[0]
    monkeypatch.setattr(bench, "screen_source_hash", lambda: h)
    assert bench._profile_traffic(1000) == per_row * 1000
    monkeypatch.setattr(bench, "screen_source_hash", lambda: "0" * 16)
    assert bench._profile_traffic(1000) is None


def test_direct_kernel_name_follows_the_launcher():
    """The roofline line names the direct-formula kernel the library runs for
    the shape: small d with C in shared memory, the tiled FP32 kernel for
    16 <= d <= 128 with d % 4 == 0, one thread per row otherwise, FP64 alone."""
    import bench
    assert bench._direct_kernel_name("fp32", 5, 16) == "k_direct_small<5>"
    assert bench._direct_kernel_name("fp32", 8, 2048) == "k_direct_assign<float>"  # C over 32 KB
    assert bench._direct_kernel_name("fp32", 128, 1024) == "k_direct_tiled"
    assert bench._direct_kernel_name("fp32", 130, 64) == "k_direct_assign<float>"
    assert bench._direct_kernel_name("fp64", 5, 16) == "k_direct_assign<double>"
