"""Host-side checks of the C-ABI library that need no GPU.

* the library loads and exports every function include/ifdk.h declares;
* argument validation happens before any device work;
* the fold kernel's TMA boxes contain every tap of every thread: the kernel's
  window and tap arithmetic is emulated (FP64 on the FP32 terms) for every
  block and view of the parity geometries and sampled blocks of the large
  ones, against the box sizes the library itself chooses
  (``ifdk_query_backproject``).  This runs before any kernel touches a GPU.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1909_02724_gb300 import binding as B
from paper_1909_02724_gb300.build import INCLUDE, LIB, build
from paper_1909_02724_gb300.geometry import circular
from paper_1909_02724_gb300.phantom import scaled_geometry, workload

TILE, PAIRS, MARGIN = 16, 16, 1


@pytest.fixture(scope="module", autouse=True)
def built():
    build()


def test_exports_every_declared_symbol():
    decl = set()
    for f in os.listdir(INCLUDE):
        if f.endswith(".h"):
            txt = open(os.path.join(INCLUDE, f)).read()
            decl |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ifdk_\w+)\s*\(", txt, re.M))
    assert decl == set(B.EXPORTS)
    lib = ctypes.CDLL(LIB)
    for name in decl:
        assert hasattr(lib, name), name


def test_status_strings_and_validation():
    assert B.status_string(B.IFDK_OK) == "ok"
    assert "aligned" in B.status_string(B.IFDK_ERR_ALIGNMENT)
    g = scaled_geometry(16, 16, 8)
    bad = [g.with_(nu=0), g.with_(dx=-1.0), g.with_(sdd=500.0), g.with_(nx=2000, ny=2000),
           g.with_(angles=np.array([np.nan] * 8))]
    for b in bad:
        with pytest.raises(B.IfdkError) as e:
            B.ifdk_create(b)
        assert e.value.code in (B.IFDK_ERR_INVALID, B.IFDK_ERR_GEOMETRY)


def _f32(x):
    return np.float32(x).astype(np.float64)


def _terms(g):
    """FP32 per-view terms as the plan forms them (FP64 closed form, cast)."""
    cb, sb = np.cos(g.angles), np.sin(g.angles)
    return dict(C0=_f32(g.dx * sb), C1=_f32(-g.dy * cb), C3=_f32(np.full_like(cb, g.sid)),
                A0=_f32(g.sdd * g.dx * cb / g.du), A1=_f32(g.sdd * g.dy * sb / g.du),
                B2=_f32(np.full_like(cb, g.sdd * g.dz / g.dv)))


def check_fold_windows(g, q_dtype, blocks=None):
    info = B.ifdk_query_backproject(g, q_dtype)
    if info["path"] != 1:
        return info
    H, BW, FW, AL = info["box_h"], info["box_w"], info["fold_w"], info["align"]
    t = _terms(g)
    cx, cy, cz = (g.nx - 1) / 2, (g.ny - 1) / 2, (g.nz - 1) / 2
    uc, vc = (g.nu - 1) / 2 + g.off_u / g.du, (g.nv - 1) / 2 + g.off_v / g.dv
    tiles_x, tiles_y = -(-g.nx // TILE), -(-g.ny // TILE)
    zblocks = -(-((g.nz + 1) // 2) // PAIRS)
    if blocks is None:
        blocks = [(bx, by, bz) for bx in range(tiles_x) for by in range(tiles_y) for bz in range(zblocks)]
    tx, ty = np.meshgrid(np.arange(TILE), np.arange(TILE), indexing="ij")
    tx, ty = tx.ravel(), ty.ravel()
    p = np.arange(PAIRS)
    V = slice(None)
    for bx, by, bz in blocks:
        i0, j0, k0 = bx * TILE, by * TILE, bz * PAIRS
        kp0 = k0 - cz
        ia, ib, ja, jb = i0 - cx, i0 + TILE - 1 - cx, j0 - cy, j0 + TILE - 1 - cy
        ci, cj = np.array([ia, ib, ia, ib]), np.array([ja, ja, jb, jb])
        zc = t["C0"][:, None] * ci + t["C1"][:, None] * cj + t["C3"][:, None]
        ucn = (t["A0"][:, None] * ci + t["A1"][:, None] * cj) / zc
        u_lo, z_lo, z_hi = ucn.min(1), zc.min(1), zc.max(1)
        e0, e1 = t["B2"] * kp0, t["B2"] * (kp0 + PAIRS - 1)
        v_lo = np.minimum(np.minimum(e0 / z_lo, e0 / z_hi), np.minimum(e1 / z_lo, e1 / z_hi))
        u0f = np.floor(uc + u_lo) - MARGIN
        u0a = np.floor(u0f / AL) * AL
        off = u0f - u0a
        v0 = np.floor(vc + v_lo) - MARGIN
        assert off.min() >= 0 and (off + FW).max() <= BW - 1
        # every thread / pair of the block (masked threads included)
        ip = (i0 + tx) - cx
        jp = (j0 + ty) - cy
        z = t["C0"][V, None] * ip + t["C1"][V, None] * jp + t["C3"][V, None]
        f = 1.0 / z
        ul = (t["A0"][V, None] * ip + t["A1"][V, None] * jp) * f + (uc - u0f)[:, None]
        assert ul.min() >= 0.01 and ul.max() < FW - 0.01, (bx, by, bz, ul.min(), ul.max(), FW)
        sig = t["B2"][:, None] * f
        vl = (vc - v0)[:, None, None] + sig[:, :, None] * (kp0 + p)[None, None, :]
        assert vl.min() >= 0.01 and vl.max() < H - 1 - 0.01, (bx, by, bz, vl.min(), vl.max(), H)
    return info


@pytest.mark.parametrize("dtype", [B.IFDK_F32, B.IFDK_F16, B.IFDK_BF16])
@pytest.mark.parametrize("geom", [
    scaled_geometry(64, 64, 64),
    scaled_geometry(40, 56, 24, nz=50, n_det_v=48),
    scaled_geometry(33, 48, 16, nz=33),
    circular(12, 64, 48, 1.5, 1.5, 37, 29, 21, 1.0, sid=1000.0, sdd=1500.0, off_u=0.6, off_v=0.75),
    circular(10, 16, 16, 1.4, 1.3, 8, 8, 8, 1.1, 1.0, 0.9, sid=60.0, sdd=95.0, start=0.3),
])
def test_fold_windows_contain_every_tap(geom, dtype):
    check_fold_windows(geom, dtype)


@pytest.mark.parametrize("name", ["fdk64", "grad32"])
def test_fold_windows_small_workloads(name):
    for dt in (B.IFDK_F32, B.IFDK_F16):
        assert check_fold_windows(workload(name).geom, dt)["path"] == 1


@pytest.mark.parametrize("name", ["fdk512", "grad256", "fdk2048", "slab4096"])
def test_fold_windows_large_workloads(name):
    g = workload(name).geom
    tiles_x, tiles_y = -(-g.nx // TILE), -(-g.ny // TILE)
    zb = -(-((g.nz + 1) // 2) // PAIRS)
    rng = np.random.default_rng(0)
    blocks = {(0, 0, 0), (tiles_x - 1, tiles_y - 1, zb - 1), (tiles_x // 2, tiles_y // 2, zb // 2),
              (0, tiles_y - 1, 0), (tiles_x - 1, 0, zb - 1)}
    blocks |= {(int(rng.integers(tiles_x)), int(rng.integers(tiles_y)), int(rng.integers(zb))) for _ in range(6)}
    if g.np > 512:   # subsample views for the largest scans
        g = g.with_(angles=g.angles[::4])
    for dt in (B.IFDK_F32, B.IFDK_F16):
        info = check_fold_windows(g, dt, sorted(blocks))
        assert info["path"] == 1, (name, dt, info)


def test_general_path_for_offcentre_and_fractional_centre():
    g = scaled_geometry(32, 48, 8)
    assert B.ifdk_query_backproject(g, B.IFDK_F32)["path"] == 1
    assert B.ifdk_query_backproject(g.with_(vol_off_z=1.0), B.IFDK_F32)["path"] == 0
    assert B.ifdk_query_backproject(g.with_(off_v=0.3 * g.dv), B.IFDK_F32)["path"] == 0
    assert B.ifdk_query_backproject(g.with_(off_v=0.5 * g.dv), B.IFDK_F32)["path"] == 1
    assert B.ifdk_query_backproject(g.with_(nu=50), B.IFDK_F16)["path"] == 0   # rows not 16-byte multiples


def _gpu_test_geoms():
    import importlib
    return importlib.import_module("tests.test_gpu_parity").GEOMS


@pytest.mark.parametrize("dtype", [B.IFDK_F32, B.IFDK_F16, B.IFDK_BF16])
def test_fold_windows_of_every_gpu_test_geometry(dtype):
    for name, g in _gpu_test_geoms().items():
        check_fold_windows(g, dtype)


# ---------------------------------------------------------------------------
# Packed views: the packed kernel's windows (emulated like the fold kernel's)
# hold every tap, and every tap row a written voxel reads is a packed row
# unless both it and its mirror lie outside the detector (then 0 is right).

TAIL_L = 4   # z pairs of the packed kernel's tail blocks


def packed_zblocks(npairs, L):
    """z-blocks of a packed launch: npairs // L blocks of L pairs, then the
    remainder in blocks of TAIL_L pairs."""
    return npairs // L + -(-(npairs % L) // TAIL_L)


def check_packed_windows(g, q_dtype, view_pairing=True, blocks=None, pair0=0, pcount=None):
    info = B.ifdk_query_packed(g, q_dtype, view_pairing)
    if info["path"] == 0:
        return info
    H, BW, L, AL = info["box_h"], info["box_w"], info["z_per_thread"], info["align"]
    r0, R = info["row0"], info["rows"]
    t = _terms(g)
    cx, cy, cz = (g.nx - 1) / 2, (g.ny - 1) / 2, (g.nz - 1) / 2
    uc, vc = (g.nu - 1) / 2 + g.off_u / g.du, (g.nv - 1) / 2 + g.off_v / g.dv
    two_vc = int(round(2 * vc))
    ny_cols = g.ny // 2 if info["path"] in (2, 4) else g.ny
    nx_cols = g.nx // 2 if info["path"] == 4 else g.nx
    tiles_x, tiles_y = -(-nx_cols // TILE), -(-ny_cols // TILE)
    npairs = (g.nz + 1) // 2
    if pcount is None:
        zblocks = packed_zblocks(npairs, L)
        assert info["blocks"] == tiles_x * tiles_y * zblocks
        pcount = npairs
    else:
        zblocks = packed_zblocks(pcount, L)       # a pair-range launch
    if blocks is None:
        blocks = [(bx, by, bz) for bx in range(tiles_x) for by in range(tiles_y) for bz in range(zblocks)]
    tx, ty = np.meshgrid(np.arange(TILE), np.arange(TILE), indexing="ij")
    tx, ty = tx.ravel(), ty.ravel()
    zfull = pcount // L
    for bx, by, bz in blocks:
        # full z-blocks of L pairs, then tail blocks of TAIL_L pairs, from pair pair0 on
        Lb = L if bz < zfull else TAIL_L
        k0 = pair0 + (bz * L if bz < zfull else zfull * L + (bz - zfull) * TAIL_L)
        p = np.arange(Lb)
        i0, j0 = bx * TILE, by * TILE
        kp0 = k0 - cz
        ia, ib, ja, jb = i0 - cx, i0 + TILE - 1 - cx, j0 - cy, j0 + TILE - 1 - cy
        ci, cj = np.array([ia, ib, ia, ib]), np.array([ja, ja, jb, jb])
        zc = t["C0"][:, None] * ci + t["C1"][:, None] * cj + t["C3"][:, None]
        ucn = (t["A0"][:, None] * ci + t["A1"][:, None] * cj) / zc
        u_lo, z_lo, z_hi = ucn.min(1), zc.min(1), zc.max(1)
        e0, e1 = t["B2"] * kp0, t["B2"] * (kp0 + Lb - 1)
        v_lo = np.minimum(np.minimum(e0 / z_lo, e0 / z_hi), np.minimum(e1 / z_lo, e1 / z_hi))
        u0a = np.floor((np.floor(uc + u_lo) - MARGIN + 1) / AL) * AL - 1
        # the TMA box starts at element u0a + 1: 4 values of q_dtype each, 16-byte aligned
        assert np.all((4 * (u0a + 1) * (4 if q_dtype == B.IFDK_F32 else 2)) % 16 == 0)
        v0 = np.floor(vc + v_lo) - MARGIN
        ip = (i0 + tx) - cx
        jp = (j0 + ty) - cy
        z = t["C0"][:, None] * ip + t["C1"][:, None] * jp + t["C3"][:, None]
        f = 1.0 / z
        ul = (t["A0"][:, None] * ip + t["A1"][:, None] * jp) * f + (uc - u0a)[:, None]
        # element cu = floor(ul) holds columns cu and cu + 1
        assert ul.min() >= 0.01 and ul.max() < BW - 0.01, (bx, by, bz, ul.min(), ul.max(), BW)
        sig = t["B2"][:, None] * f
        vl = (vc - v0)[:, None, None] + sig[:, :, None] * (kp0 + p)[None, None, :]
        # box containment of every pair the block computes, written or not: a tail block
        # runs all Lb pairs, up to Lb - 1 of them past pair0 + pcount (or past the middle)
        assert vl.shape[-1] == Lb
        assert vl.min() >= 0.01 and vl.max() < H - 1 - 0.01, (bx, by, bz, vl.min(), vl.max(), H)
        # packed element u0a + floor(ul) (column c = element - 1 + 1 ... held from column -1 on)
        cols = u0a[:, None] + np.floor(ul)
        c_in = (cols >= -1) & (cols < -1 + info["row_elems"])
        c_off = (cols + 1 < 0) | (cols >= g.nu)          # both taps c, c + 1 off the detector
        assert np.all(c_in | c_off), (bx, by, bz)
        # the detector rows behind the taps of the pairs that are written must be packed rows
        # (a discarded pair's taps only have to stay inside the box, checked above)
        written = (k0 + p) < pair0 + pcount
        rows = v0[:, None, None] + np.floor(vl[:, :, written])
        for rr in (rows, rows + 1):
            inside = (rr >= r0) & (rr < r0 + R)
            off_det = ((rr < 0) | (rr >= g.nv)) & ((two_vc - rr < 0) | (two_vc - rr >= g.nv))
            assert np.all(inside | off_det), (bx, by, bz)
    return info


@pytest.mark.parametrize("dtype", [B.IFDK_F32, B.IFDK_F16, B.IFDK_BF16])
@pytest.mark.parametrize("geom", [
    scaled_geometry(64, 64, 64),
    scaled_geometry(40, 56, 24, nz=50, n_det_v=48),
    scaled_geometry(33, 48, 16, nz=33),
    circular(10, 64, 48, 1.5, 1.5, 36, 28, 22, 1.0, off_u=-0.4, off_v=0.75),
    circular(10, 64, 48, 1.5, 1.5, 36, 28, 22, 1.0, off_u=0.2, off_v=-0.75),
    circular(12, 64, 48, 1.5, 1.5, 36, 28, 22, 1.0, off_v=-4.5),
    circular(9, 96, 80, 0.5, 0.5, 24, 24, 20, 0.5),
])
def test_packed_windows_contain_every_tap(geom, dtype):
    for pairing in (True, False):
        info = check_packed_windows(geom, dtype, view_pairing=pairing)
        assert info["path"] == (2 if pairing and geom.ny % 2 == 0 and geom.np % 2 == 0 else 1)


@pytest.mark.parametrize("geom", [
    scaled_geometry(64, 64, 64),
    scaled_geometry(48, 64, 40, nz=42),
    scaled_geometry(32, 48, 16, nz=33),
    circular(12, 64, 48, 1.5, 1.5, 36, 36, 22, 1.0, off_u=-0.4, off_v=-4.5),
])
def test_quad_windows_contain_every_tap(geom):
    """Quarter-turn quads (FP16 storage): the quadrant's tiles and every view."""
    info = check_packed_windows(geom, B.IFDK_F16, view_pairing=2)
    assert info["path"] == 4
    assert B.ifdk_query_packed(geom, B.IFDK_F32, 2)["path"] == 2      # quads are FP16 only
    assert B.ifdk_query_packed(geom, B.IFDK_F16, 1)["path"] == 2


def test_quad_windows_random_square_geometries():
    """Seeded square geometries (quads apply): whole-volume and random pair-range
    launches keep every tap of every block in its window."""
    from tests.random_geometries import random_square_geometries
    rng = np.random.default_rng(9)
    for _, g in random_square_geometries():
        info = check_packed_windows(g, B.IFDK_F16, view_pairing=2)
        assert info["path"] == 4
        npairs = (g.nz + 1) // 2
        pb = int(rng.integers(0, npairs))
        pc = int(rng.integers(1, npairs - pb + 1))
        check_packed_windows(g, B.IFDK_F16, 2, pair0=pb, pcount=pc)


def test_quad_detection():
    """Path 4 needs np % 4 == 0 with exact quarter turns and a square, even column grid."""
    g = scaled_geometry(32, 48, 16)
    assert B.ifdk_query_packed(g, B.IFDK_F16, 2)["path"] == 4
    assert B.ifdk_query_packed(g.with_(angles=g.angles[:14]), B.IFDK_F16, 2)["path"] in (1, 2)  # np % 4 != 0
    assert B.ifdk_query_packed(g.with_(ny=30), B.IFDK_F16, 2)["path"] == 2            # not square
    assert B.ifdk_query_packed(g.with_(dy=g.dx * 1.01), B.IFDK_F16, 2)["path"] == 2   # pitches differ
    six = circular(18, 48, 48, 96 / 48, 96 / 48, 32, 32, 32, 2.0)                    # 18 views: no quarter turn
    assert B.ifdk_query_packed(six, B.IFDK_F16, 2)["path"] == 2
    jitter = g.angles.copy()
    jitter[g.np // 4 + 1] += 1e-6
    jitter[3 * g.np // 4 + 1] += 1e-6                                                # half turns still exact
    assert B.ifdk_query_packed(g.with_(angles=jitter), B.IFDK_F16, 2)["path"] == 2


def test_packed_path_declines_wide_footprints():
    """A strongly magnified scan (window wider than the largest box) has no
    packed path; ifdk_backproject's general kernel serves it."""
    g = circular(6, 16, 16, 1.4, 1.3, 8, 8, 8, 1.1, 1.0, 0.9, sid=60.0, sdd=95.0, start=0.3)
    assert B.ifdk_query_packed(g, B.IFDK_F32)["path"] == 0
    assert B.ifdk_query_backproject(g, B.IFDK_F32)["path"] == 0


@pytest.mark.parametrize("name", ["fdk512", "grad256", "fdk2048", "slab4096"])
def test_packed_windows_large_workloads(name):
    g = workload(name).geom
    rng = np.random.default_rng(1)
    if g.np > 512:   # subsample views for the largest scans
        g = g.with_(angles=g.angles[::4])
    for dt in (B.IFDK_F32, B.IFDK_F16):
        for pairing in (True, False):
            info = B.ifdk_query_packed(g, dt, pairing)
            ny_cols = g.ny // 2 if info["path"] == 2 else g.ny
            tx, ty = -(-g.nx // TILE), -(-ny_cols // TILE)
            zb = packed_zblocks((g.nz + 1) // 2, info["z_per_thread"])
            blocks = {(0, 0, 0), (tx - 1, ty - 1, zb - 1), (tx // 2, ty // 2, zb // 2), (0, ty - 1, 0),
                      (tx - 1, 0, zb - 1)}
            blocks |= {(int(rng.integers(tx)), int(rng.integers(ty)), int(rng.integers(zb))) for _ in range(6)}
            info = check_packed_windows(g, dt, pairing, sorted(blocks))
            assert info["path"] == (2 if pairing else 1), (name, dt, info)


def test_half_turn_pairing_detection():
    """Path 2 (half-turn view pairs) exactly when every view s < np/2 has a
    partner s + np/2 turned by pi and ny is even; otherwise single views."""
    g = scaled_geometry(32, 48, 16)
    assert B.ifdk_query_packed(g, B.IFDK_F32)["path"] == 2
    assert B.ifdk_query_packed(g, B.IFDK_F32, view_pairing=False)["path"] == 1
    assert B.ifdk_query_packed(g.with_(ny=31), B.IFDK_F32)["path"] == 1                  # odd ny
    odd = circular(15, 48, 48, 96 / 48, 96 / 48, 32, 32, 32, 2.0)
    assert B.ifdk_query_packed(odd, B.IFDK_F32)["path"] == 1                              # odd np
    short = g.with_(angles=np.linspace(0, np.pi + 0.4, g.np, endpoint=False))
    assert B.ifdk_query_packed(short, B.IFDK_F32)["path"] == 1                            # no partner at +pi
    jitter = g.angles.copy()
    jitter[g.np // 2 + 3] += 1e-6
    assert B.ifdk_query_packed(g.with_(angles=jitter), B.IFDK_F32)["path"] == 1
    assert B.ifdk_query_packed(g.with_(angles=g.angles + 0.37), B.IFDK_F32)["path"] == 2   # any start angle
    # packed views need the mirror path: centred volume, 2 vc integral
    assert B.ifdk_query_packed(g.with_(vol_off_z=1.0), B.IFDK_F32)["path"] == 0
    assert B.ifdk_query_packed(g.with_(off_v=0.3 * g.dv), B.IFDK_F32)["path"] == 0


def test_packed_rows_cover_mirrors_above_the_detector():
    """r0 = min(0, 2 vc - (nv - 1)): with the principal point above the centre,
    rows above the detector whose mirrors are on it are packed too."""
    for off_px, r0 in [(0.0, 0), (0.5, 0), (-0.5, -1), (-3.0, -6)]:
        g = circular(12, 64, 48, 1.5, 1.5, 36, 28, 22, 1.0, off_v=off_px * 1.5)
        info = B.ifdk_query_packed(g, B.IFDK_F32)
        vc = (g.nv - 1) / 2 + off_px
        assert info["row0"] == r0
        assert info["rows"] == int(np.floor(vc)) + 3 - r0
        assert info["row_elems"] == g.nu + 2          # columns -1 .. nu - 1, rounded up to even


def test_packed_path_needs_row_steps_below_two():
    """The packed kernel reuses rows for steps of at most two rows per voxel:
    the plan declines scans whose largest step D dz / (dv z_min) reaches 1.9."""
    g = circular(8, 64, 64, 0.5, 0.5, 16, 16, 16, 0.5, dz=0.5)
    assert B.ifdk_query_packed(g, B.IFDK_F32)["path"] in (1, 2)      # step ~1.5
    assert B.ifdk_query_packed(g.with_(dz=0.7), B.IFDK_F32)["path"] == 0   # step ~2.1


def test_packed_windows_random_geometries():
    """Every tap of every block and view lies in its window for the seeded random
    geometries that the GPU parity sweep runs."""
    from tests.random_geometries import random_geometries
    for name, g in random_geometries():
        for dt in (B.IFDK_F32, B.IFDK_F16, B.IFDK_BF16):
            for pairing in (True, False):
                check_packed_windows(g, dt, pairing)


def test_every_entry_point_refuses_a_null_plan_before_any_cuda_call():
    """With a NULL plan (or NULL outputs) every call returns IFDK_ERR_INVALID
    without touching the device (this runs without a GPU); ifdk_destroy(NULL)
    is a no-op."""
    lib = B.load_library()
    for name in B.EXPORTS:
        if name in ("ifdk_status_string",):
            continue
        fn = getattr(lib, name)
        args = []
        for t in fn.argtypes:
            if t in (ctypes.c_int, ctypes.c_int32):
                args.append(0)
            elif t in (ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int64, ctypes.c_longlong):
                args.append(0)
            elif t in (ctypes.c_float, ctypes.c_double):
                args.append(0.0)
            else:
                args.append(None)
        rc = fn(*args)
        if name == "ifdk_destroy":
            assert rc == B.IFDK_OK
        else:
            assert rc == B.IFDK_ERR_INVALID, (name, rc)


def test_packed_windows_of_pair_ranges():
    """Pair-range launches start their z-blocks at any pair: every tap of every
    block still lies in its window."""
    from tests.random_geometries import random_geometries
    geoms = [g for _, g in random_geometries()] + [scaled_geometry(64, 64, 64), scaled_geometry(33, 48, 16, nz=33),
                                                   circular(12, 64, 48, 1.5, 1.5, 36, 28, 22, 1.0, off_v=-4.5)]
    rng = np.random.default_rng(8)
    for g in geoms:
        npairs = (g.nz + 1) // 2
        for _ in range(3):
            pb = int(rng.integers(0, npairs))
            pc = int(rng.integers(1, npairs - pb + 1))
            for dt in (B.IFDK_F32, B.IFDK_F16):
                for pairing in (True, False):
                    check_packed_windows(g, dt, pairing, pair0=pb, pcount=pc)
