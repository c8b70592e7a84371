"""Pins of the oracle's geometry, back-projection (Algorithms 2, 3) and adjoint.

The brute-force reference below derives each voxel's detector coordinates from
the scanner's world-space source and detector (ray / plane intersection), not
from the projection matrices, so a wrong sign, index or transposed operand in
the oracle's Eq. 2 product shows up as a mismatch."""
import numpy as np
import pytest

import oracle
from paper_1909_02724_gb300.geometry import circular
from paper_1909_02724_gb300.phantom import (line_integrals, pixel_positions, principal_point,
                                            random_ellipsoids, scaled_geometry, source_positions,
                                            sphere)


def voxel_world(g, i, j, k):
    """World position of voxel index (i, j, k): X right with i, Y down with j,
    Z down with k (the orientation fixed by M0), centred on the axis + vol_off_z."""
    X = g.dx * (np.asarray(i, float) - (g.nx - 1) / 2.0)
    Y = -g.dy * (np.asarray(j, float) - (g.ny - 1) / 2.0)
    Z = -g.dz * (np.asarray(k, float) - (g.nz - 1) / 2.0) + g.vol_off_z
    return np.stack(np.broadcast_arrays(X, Y, Z), -1)


def ray_uv(g, s, x):
    """Detector coordinates (u, v) and source-axis distance c of world points x,
    by intersecting the line source->x with the detector plane."""
    beta = g.angles[s]
    S = source_positions(g, [s])[0]
    uc, vc = principal_point(g)
    C = pixel_positions(g, beta, uc, vc)
    n = (C - S) / np.linalg.norm(C - S)
    eu = pixel_positions(g, beta, uc + 1.0, vc) - C
    ev = pixel_positions(g, beta, uc, vc + 1.0) - C
    c = (x - S) @ n
    hit = S + (g.sdd / c)[..., None] * (x - S)
    u = uc + (hit - C) @ eu / (g.du ** 2)
    v = vc + (hit - C) @ ev / (g.dv ** 2)
    return u, v, c


def test_matrix_maps_ray_points_to_their_pixel():
    g = scaled_geometry(12, 20, 5, n_det_v=14, nz=10).with_(off_u=0.4, off_v=-0.6, vol_off_z=1.5)
    P = oracle.projection_matrices(g)
    rng = np.random.default_rng(3)
    for s in range(g.np):
        beta = g.angles[s]
        S = source_positions(g, [s])[0]
        iu, iv = rng.uniform(0, g.nu - 1, 8), rng.uniform(0, g.nv - 1, 8)
        pix = pixel_positions(g, beta, iu, iv)
        for t in (0.55, 0.66, 0.7):
            x = S + t * (pix - S)
            i = x[:, 0] / g.dx + (g.nx - 1) / 2.0
            j = -x[:, 1] / g.dy + (g.ny - 1) / 2.0
            k = -(x[:, 2] - g.vol_off_z) / g.dz + (g.nz - 1) / 2.0
            h = P[s] @ np.stack([i, j, k, np.ones_like(i)])
            np.testing.assert_allclose(h[0] / h[2], iu, atol=1e-9)
            np.testing.assert_allclose(h[1] / h[2], iv, atol=1e-9)
            # homogeneous z = distance of the point from the source along the central ray
            _, _, c = ray_uv(g, s, x)
            np.testing.assert_allclose(h[2], c, rtol=1e-12)


def test_eq3_and_theorems():
    """Eq. 3 (z printed in the paper), Theorem 2/3 (u, z independent of k) and
    Theorem 1 (v(k) + v(Nz-1-k) = Nv - 1 for a centred volume and detector)."""
    g = scaled_geometry(10, 16, 7, nz=9)
    P = oracle.projection_matrices(g)
    i, j = np.meshgrid(np.arange(g.nx), np.arange(g.ny), indexing="ij")
    for s, beta in enumerate(g.angles):
        assert abs(P[s][0][2]) < 1e-12 and abs(P[s][2][2]) < 1e-12
        z = P[s][2][0] * i + P[s][2][1] * j + P[s][2][3]
        eq3 = g.sid + np.sin(beta) * (i - (g.nx - 1) / 2) * g.dx - np.cos(beta) * (j - (g.ny - 1) / 2) * g.dy
        np.testing.assert_allclose(z, eq3, rtol=1e-14)
        for k in range(g.nz):
            t1 = P[s] @ np.array([3.0, 5.0, k, 1.0])
            t2 = P[s] @ np.array([3.0, 5.0, g.nz - 1 - k, 1.0])
            assert abs(t1[1] / t1[2] + t2[1] / t2[2] - (g.nv - 1)) < 1e-10


def test_view_weights():
    g = scaled_geometry(4, 4, 12)
    np.testing.assert_allclose(oracle.view_weights(g), 2 * np.pi / 12, rtol=1e-14)
    g2 = g.with_(angles=np.sort(np.random.default_rng(0).uniform(0, 2 * np.pi, 9)))
    assert oracle.view_weights(g2).sum() == pytest.approx(2 * np.pi, rel=1e-12)
    g3 = g.with_(angles=-g.angles)                       # clockwise scan, same weights
    np.testing.assert_allclose(oracle.view_weights(g3), 2 * np.pi / 12, rtol=1e-12)


def brute_force_bp_of_impulse(g, s, r, c):
    """Back-projection of a unit impulse at pixel (r, c) of view s, every voxel:
    fdk weight * (1/c^2) * hat(u - c) * hat(v - r)."""
    ii, jj, kk = np.meshgrid(np.arange(g.nx), np.arange(g.ny), np.arange(g.nz), indexing="ij")
    x = voxel_world(g, ii, jj, kk)
    u, v, dist = ray_uv(g, s, x)
    hat = lambda t: np.maximum(0.0, 1.0 - np.abs(t))  # noqa: E731
    w = oracle.view_weights(g)[s] * g.sid * g.sdd / (2.0 * g.du)
    return w / dist ** 2 * hat(u - c) * hat(v - r)


@pytest.mark.parametrize("offsets", [(0.0, 0.0, 0.0), (0.35, -0.8, 0.6)])
def test_brute_force_8cube(offsets):
    g = circular(5, 10, 9, 1.4, 1.3, 8, 8, 8, 1.1, 1.0, 0.9, sid=60.0, sdd=95.0, start=0.3)
    g = g.with_(off_u=offsets[0], off_v=offsets[1], vol_off_z=offsets[2])
    rng = np.random.default_rng(7)
    for _ in range(12):
        s, r, c = int(rng.integers(g.np)), int(rng.integers(g.nv)), int(rng.integers(g.nu))
        Q = np.zeros((g.np, g.nv, g.nu))
        Q[s, r, c] = 1.0
        got = oracle.backproject(g, Q)
        expect = brute_force_bp_of_impulse(g, s, r, c)
        assert np.max(np.abs(got - expect)) <= 1e-12 * max(1.0, np.max(np.abs(expect)))
        # the adjoint of the same matrix: project(e_voxel) at pixel (s, r, c) = B[voxel, pixel]
        vox = tuple(int(t) for t in np.unravel_index(np.argmax(expect), expect.shape))
        x = np.zeros((g.nx, g.ny, g.nz))
        x[vox] = 1.0
        assert oracle.project(g, x)[s, r, c] == pytest.approx(expect[vox], rel=1e-12, abs=1e-300)
        assert expect.max() > 0


def test_adjoint_dot_product():
    g = circular(7, 23, 17, 1.2, 1.1, 13, 11, 9, 1.0, 1.1, 1.2, sid=80.0, sdd=130.0, off_u=0.3,
                 off_v=0.2)
    rng = np.random.default_rng(11)
    q = rng.normal(size=(g.np, g.nv, g.nu))
    x = rng.normal(size=(g.nx, g.ny, g.nz))
    lhs = float(np.sum(oracle.backproject(g, q) * x))
    rhs = float(np.sum(q * oracle.project(g, x)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


def test_rotation_by_a_quarter_turn():
    """Shifting the views by Np/4 (beta -> beta + pi/2) rotates the volume by 90 degrees
    about Z: vol'[i][j] = vol[N-1-j][i] (from the M0 index flips and Rz(beta))."""
    g = scaled_geometry(16, 24, 8, nz=6)
    rng = np.random.default_rng(2)
    Q = rng.normal(size=(g.np, g.nv, g.nu))
    v0 = oracle.backproject(g, Q)
    v1 = oracle.backproject(g, np.roll(Q, -g.np // 4, axis=0))
    np.testing.assert_allclose(v1, np.rot90(v0, -1, axes=(0, 1)), rtol=1e-11, atol=1e-11 * np.abs(v0).max())


def test_z_mirror_symmetry():
    """Up-down symmetric projections (Theorem 1) back-project to a z-symmetric volume."""
    g = scaled_geometry(10, 20, 6, n_det_v=15, nz=7)
    rng = np.random.default_rng(4)
    Q = rng.normal(size=(g.np, g.nv, g.nu))
    Q = Q + Q[:, ::-1, :]
    vol = oracle.backproject(g, Q)
    np.testing.assert_allclose(vol, vol[:, :, ::-1], rtol=1e-12, atol=1e-12 * np.abs(vol).max())


@pytest.mark.parametrize("n,tol", [(64, 5e-3), (128, 1e-3)])
def test_uniform_sphere_centre(n, tol):
    """FDK of a uniform ball of density 1 (radius 20 mm) is 1 at the centre up to cone-beam
    and discretisation error: pins the cosine weight, ramp scale and FDK constant."""
    g = scaled_geometry(n, n, n)
    if n == 128:
        g = g.with_(nz=2)                                 # mid-plane only
    E = line_integrals(sphere(20.0), g)
    vol = oracle.fdk(g, E)
    c = g.nx // 2
    kc = g.nz // 2
    centre = vol[c - 1:c + 1, c - 1:c + 1, kc - 1:kc + 1].mean()
    assert abs(centre - 1.0) <= tol


def test_sampled_and_sparse_paths_agree_with_dense():
    g = scaled_geometry(12, 18, 9, nz=8).with_(off_v=0.25)
    E = line_integrals(random_ellipsoids(4, 5.0, seed=8), g)
    Q = oracle.filter_views(g, E)
    dense = oracle.backproject(g, Q)
    rng = np.random.default_rng(5)
    vox = np.stack([rng.integers(0, g.nx, 40), rng.integers(0, g.ny, 40), rng.integers(0, g.nz, 40)], 1)
    np.testing.assert_allclose(oracle.backproject_voxels(g, Q, vox), dense[vox[:, 0], vox[:, 1], vox[:, 2]],
                               rtol=0, atol=0)
    need = oracle.rows_needed(g, vox)
    s_idx, r_idx = np.nonzero(need)
    rowmap = -np.ones((g.np, g.nv), dtype=np.int64)
    rowmap[s_idx, r_idx] = np.arange(len(s_idx))
    Qs = oracle.filter_rows(g, E[s_idx, r_idx], r_idx)
    np.testing.assert_allclose(oracle.backproject_voxels(g, Qs, vox, rowmap=rowmap),
                               dense[vox[:, 0], vox[:, 1], vox[:, 2]], rtol=1e-13, atol=1e-13)
    # view ranges split and summed give the whole
    part = oracle.backproject(g, Q, 0, 4)
    oracle.backproject(g, Q, 4, g.np - 4, vol=part)
    np.testing.assert_allclose(part, dense, rtol=1e-12, atol=1e-12 * np.abs(dense).max())
