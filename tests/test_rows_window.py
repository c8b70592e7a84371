"""Detector-row windows (host logic, no GPU): ifdk_query_rows bounds the rows a
volume reads, and a plan whose detector is cut to those rows reconstructs the
same volume.  Both are checked against the FP64 oracle: every row its
bilinear taps touch lies inside the window, and its back-projection of the
cropped views equals the full one."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300 import binding as B
from paper_1909_02724_gb300.build import build
from paper_1909_02724_gb300.geometry import circular
from paper_1909_02724_gb300.phantom import scaled_geometry, workload


@pytest.fixture(scope="module", autouse=True)
def built():
    build()


def all_voxels(g):
    ii, jj, kk = np.meshgrid(np.arange(g.nx), np.arange(g.ny), np.arange(g.nz), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1)


GEOMS = {
    "slab": scaled_geometry(32, 48, 24, nz=8),                          # central slab, mirror path
    "offcentre": scaled_geometry(24, 40, 16, nz=6).with_(vol_off_z=9.0),  # slab above the source plane
    "detoffset": circular(12, 40, 64, 1.5, 1.0, 16, 16, 12, 1.0, off_v=3.7, off_u=-2.0),
    "thick": scaled_geometry(16, 32, 8, nz=16),
}


@pytest.mark.parametrize("name", list(GEOMS))
def test_window_contains_every_row_the_oracle_touches(name):
    g = GEOMS[name]
    r0, n = B.ifdk_query_rows(g)
    need = oracle.rows_needed(g, all_voxels(g))
    rows = np.nonzero(need.any(axis=0))[0]
    assert len(rows) > 0 and n > 0
    assert r0 <= rows.min() and rows.max() < r0 + n, (name, r0, n, rows.min(), rows.max())
    assert n <= rows.max() - rows.min() + 1 + 4          # tight: at most two spare rows per side
    # a view subset reads a subset of the rows
    s0, sn = B.ifdk_query_rows(g, 3, 5)
    sub = np.nonzero(oracle.rows_needed(g, all_voxels(g))[3:8].any(axis=0))[0]
    assert s0 <= sub.min() and sub.max() < s0 + sn


def test_window_of_the_slab_workload():
    """4096x4096x256 central slab from a 4096-row detector reads ~270 rows."""
    g = workload("slab4096").geom
    r0, n = B.ifdk_query_rows(g)
    assert 250 <= n <= 300
    assert abs((r0 + (n - 1) / 2) - (g.nv - 1) / 2) <= 1        # centred on the principal row
    assert B.ifdk_query_rows(g.crop_rows(r0, n)) == (0, n)        # the cut plan needs all of its rows


def test_rows_query_edge_cases():
    g = GEOMS["slab"]
    assert B.ifdk_query_rows(g, 0, 0) == (0, 0)
    with pytest.raises(B.IfdkError):
        B.ifdk_query_rows(g, 20, 10)                              # past the last view
    with pytest.raises(B.IfdkError):
        B.ifdk_query_rows(g, -1, 2)
    # a volume far above the detector's field of view reads no row
    far = g.with_(vol_off_z=200.0)
    assert B.ifdk_query_rows(far)[1] == 0


@pytest.mark.parametrize("name", ["slab", "offcentre", "detoffset"])
def test_cropped_plan_reconstructs_the_same_volume(name):
    g = GEOMS[name]
    r0, n = B.ifdk_query_rows(g)
    gc = g.crop_rows(r0, n)
    assert np.allclose(oracle.cosine_weight(gc), oracle.cosine_weight(g)[r0:r0 + n], rtol=0, atol=1e-15)
    Q = np.random.default_rng(7).normal(size=(g.np, g.nv, g.nu))
    full = oracle.backproject(g, Q)
    cut = oracle.backproject(gc, np.ascontiguousarray(Q[:, r0:r0 + n]))
    assert np.max(np.abs(cut - full)) <= 1e-12 * np.max(np.abs(full))


def test_crop_rejects_windows_outside_the_detector():
    g = GEOMS["slab"]
    for r0, n in ((-1, 4), (0, 0), (g.nv - 2, 3)):
        with pytest.raises(ValueError):
            g.crop_rows(r0, n)
