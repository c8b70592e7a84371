"""bench.py's host-side helpers: the clock record parsed from nvidia-smi samples
(the throttle reasons that reject a run) and the match of a committed ncu
summary to the current kernel source."""
import hashlib
import json
import os
import sys

import numpy as np

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
    for name in ("bp_packed_fdk512_f32", "bp_packed_fdk512_f16", "bp_packed_fdk2048_f32", "bp_packed_fdk2048_f16",
                 "bp_packed_fdk2048_bf16", "bp_packed_fdk2048_f16_quads"):
        rec = json.load(open(os.path.join(ROOT, "profiles", f"{name}.json")))
        got = bench.profile_record("ifdk_bp_packed.cu", name)
        if rec["source_sha1"] == hashlib.sha1(src).hexdigest():
            assert got["dram_bytes_per_launch"] == rec["dram_bytes_per_launch"] and "ncu" in got
        else:
            assert got == {}
    assert bench.profile_record("ifdk_bp_packed.cu", "no_such_profile") == {}


def test_path_ceilings_from_rates():
    """The arithmetic ceilings follow from the measured rates: with one FP32 FMA per lane
    and clock (128 lanes) and no faster packed form, the ten-op ceiling is the
    nominal 128-lane one; FP16 and BF16 paths get their instruction mixes."""
    r = {"ffma": {"lane_ops_per_clk_sm": 128.0}, "ffma2": {"lane_ops_per_clk_sm": 128.0},
         "hfma2": {"lane_ops_per_clk_sm": 256.0}, "fma_f32_f16": {"lane_ops_per_clk_sm": 128.0},
         "lop3": {"lane_ops_per_clk_sm": 64.0}, "fma_f32_bf16": {"lane_ops_per_clk_sm": 128.0}}
    c = bench.path_ceilings(r, 152, 2.07e9)
    nominal = 152 * 128 * 2.07e9 / 10 / 2 ** 30
    assert abs(c["alu10"] - nominal) < 1e-9 * nominal and abs(c["f32"] - nominal) < 1e-9 * nominal
    assert abs(c["updates_per_clk_sm"]["f16"] - 1.0 / (3 / 128 + 6 / 256 + 1 / 128)) < 1e-12
    assert abs(c["updates_per_clk_sm"]["bf16"] - 1.0 / (8 / 128 + 2 / 128)) < 1e-12
    r["ffma2"]["lane_ops_per_clk_sm"] = 256.0           # a packed FMA that doubles the lane rate
    assert abs(bench.path_ceilings(r, 152, 2.07e9)["alu10"] - 2 * nominal) < 1e-9 * nominal


def test_midplane_rows_cover_every_tap_of_the_sample():
    import oracle
    from paper_1909_02724_gb300.phantom import scaled_geometry
    g = scaled_geometry(64, 96, 24)
    vox = bench.midplane_sample(g, 3000, 7)
    assert set(vox[:, 2]) <= {g.nz // 2 - 1, g.nz // 2} and len(np.unique(vox, axis=0)) == len(vox)
    s_idx, r_idx = bench.midplane_rows(g)
    band = np.zeros((g.np, g.nv), dtype=bool)
    band[s_idx, r_idx] = True
    need = oracle.rows_needed(g, vox)
    assert not (need & ~band).any()
