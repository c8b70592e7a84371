"""Seeded random scanner geometries shared by the CPU window checks and the
GPU parity sweep (geometry parameters only; no reconstruction arithmetic)."""
import numpy as np

from paper_1909_02724_gb300.geometry import circular


def random_geometries(n=12, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nu = int(rng.integers(16, 72))
        nv = int(rng.integers(12, 64))
        du = float(rng.uniform(0.6, 1.8))
        dv = float(rng.uniform(0.6, 1.8))
        sid = float(rng.uniform(400.0, 1200.0))
        sdd = sid * float(rng.uniform(1.2, 2.0))
        nx, ny, nz = (int(rng.integers(4, 40)) for _ in range(3))
        # voxels sized so that the volume stays inside the untruncated field of view
        fov = 0.5 * min(nu * du, nv * dv) * sid / sdd
        dx = float(rng.uniform(0.4, 1.0)) * fov / max(nx, ny, nz)
        n_views = int(rng.integers(3, 40))
        # half of them with offsets: a V offset of whole half pixels keeps 2 v_c integral
        kw = {}
        if i % 2:
            kw["off_u"] = float(rng.uniform(-2.0, 2.0)) * du
            kw["off_v"] = 0.5 * int(rng.integers(-6, 7)) * dv
        if i % 4 == 3:
            kw["vol_off_z"] = float(rng.uniform(-2.0, 2.0)) * dx
        g = circular(n_views, nu, nv, du, dv, nx, ny, nz, dx, sid=sid, sdd=sdd,
                     start=float(rng.uniform(0, 2 * np.pi)), **kw)
        out.append((f"rand{i}", g))
    return out


def random_square_geometries(n=6, seed=4096):
    """Seeded geometries that admit quarter-turn view quads: square, even column
    grids with equal pitches and a view count that is a multiple of 4 (random
    detector, distances, offsets, start angle, odd or even nz)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nu = int(rng.integers(24, 80))
        nv = int(rng.integers(16, 64))
        du = float(rng.uniform(0.7, 1.6))
        dv = float(rng.uniform(0.7, 1.6))
        sid = float(rng.uniform(400.0, 1200.0))
        sdd = sid * float(rng.uniform(1.2, 1.8))
        nxy = 2 * int(rng.integers(4, 20))
        nz = int(rng.integers(4, 40))
        fov = 0.5 * min(nu * du, nv * dv) * sid / sdd
        dx = float(rng.uniform(0.4, 0.9)) * fov / max(nxy, nz)
        n_views = 4 * int(rng.integers(2, 12))
        kw = {"off_u": float(rng.uniform(-2.0, 2.0)) * du, "off_v": 0.5 * int(rng.integers(-6, 7)) * dv} if i % 2 else {}
        g = circular(n_views, nu, nv, du, dv, nxy, nxy, nz, dx, sid=sid, sdd=sdd,
                     start=float(rng.uniform(0, 2 * np.pi)), **kw)
        out.append((f"square{i}", g))
    return out
