"""bench.py's host-side helpers: the clock record parsed from nvidia-smi samples
(the throttle reasons that reject a run) and the match of a committed ncu
summary to the current kernel source."""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_samples_median_max_and_reasons():
    lines = "\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    c = bench.parse_clock_samples(lines)
    assert c["samples"] == 3 and c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    hot = lines + "\n0, 1500, 2070, 1000.0, 0x0, Not Active, Active, Not Active, Not Active"
    assert bench.parse_clock_samples(hot)["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.parse_clock_samples("")["reasons"] == ["no samples"]


def test_profile_record_matches_the_kernel_source():
    src = open(os.path.join(ROOT, "paper_1909_02724_gb300", "csrc", "ifdk_bp_packed.cu"), "rb").read()
    for dt in ("f32", "f16"):
        rec = json.load(open(os.path.join(ROOT, "profiles", f"bp_packed_fdk512_{dt}.json")))
        got = bench.profile_record("ifdk_bp_packed.cu", f"bp_packed_fdk512_{dt}")
        if rec["source_sha1"] == hashlib.sha1(src).hexdigest():
            assert got["dram_bytes_per_launch"] == rec["dram_bytes_per_launch"] and "ncu" in got
        else:
            assert got == {}
    assert bench.profile_record("ifdk_bp_packed.cu", "no_such_profile") == {}
