"""Circular cone-beam geometry parameters (Table 1 of the iFDK paper).

A plain parameter container: it holds no reconstruction arithmetic.  Lengths
are in mm, angles in radians.  The detector is ``nu`` pixels wide (U, along a
row) and ``nv`` high (V); projections are stored ``[np][nv][nu]`` (U fastest).
The volume is ``nx * ny * nz`` voxels stored ``[nx][ny][nz]`` (k fastest, the
k-major layout of Algorithm 4), centred on the rotation axis and shifted along
Z by ``vol_off_z``.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass
class Geometry:
    sid: float                 # d: source to rotation axis (mm)
    sdd: float                 # D: source to detector (mm)
    nu: int                    # detector width (pixels)
    nv: int                    # detector height (pixels)
    du: float                  # detector pitch along U (mm/pixel)
    dv: float                  # detector pitch along V (mm/pixel)
    angles: np.ndarray         # view angles beta_s (rad)
    nx: int
    ny: int
    nz: int
    dx: float                  # voxel pitch (mm/voxel)
    dy: float
    dz: float
    off_u: float = 0.0         # principal point offset from the detector centre (mm)
    off_v: float = 0.0
    vol_off_z: float = 0.0     # world Z of the volume centre (mm)
    view_weights: np.ndarray | None = field(default=None)  # per-view angular weights (rad)
    short_scan: bool = False   # Parker redundancy weights (scan over pi + 2 delta)

    def __post_init__(self):
        self.angles = np.ascontiguousarray(np.asarray(self.angles, dtype=np.float64).reshape(-1))
        if self.view_weights is not None:
            self.view_weights = np.ascontiguousarray(
                np.asarray(self.view_weights, dtype=np.float64).reshape(-1))

    @property
    def np(self) -> int:
        return int(self.angles.shape[0])

    @property
    def updates(self) -> int:
        """Voxel-view updates of one full back-projection: Nx*Ny*Nz*Np."""
        return int(self.nx) * int(self.ny) * int(self.nz) * self.np

    def with_(self, **kw) -> "Geometry":
        return replace(self, **kw)

    def crop_rows(self, row_begin: int, row_count: int) -> "Geometry":
        """The same scanner with the detector cut to rows [row_begin, row_begin + row_count):
        the principal point moves by -row_begin rows, so every voxel projects onto
        the same physical pixel (and the cosine weight is unchanged)."""
        if row_count < 1 or row_begin < 0 or row_begin + row_count > self.nv:
            raise ValueError("row window outside the detector")
        off_v = self.off_v + ((self.nv - 1) / 2.0 - row_begin - (row_count - 1) / 2.0) * self.dv
        return replace(self, nv=row_count, off_v=off_v)


def circular(n_views: int, nu: int, nv: int, du: float, dv: float, nx: int, ny: int, nz: int,
             dx: float, dy: float | None = None, dz: float | None = None, sid: float = 1000.0,
             sdd: float = 1500.0, arc: float = 2.0 * np.pi, start: float = 0.0, **kw) -> Geometry:
    """Uniformly spaced views beta_s = start + arc * s / n_views."""
    angles = start + arc * np.arange(n_views, dtype=np.float64) / n_views
    return Geometry(sid=sid, sdd=sdd, nu=nu, nv=nv, du=du, dv=dv, angles=angles, nx=nx, ny=ny,
                    nz=nz, dx=dx, dy=dx if dy is None else dy, dz=dx if dz is None else dz, **kw)


def fan_half_angle(nu: int, du: float, sdd: float, off_u: float = 0.0) -> float:
    """Largest |gamma| = |atan((u - u_c) Du / D)| over the detector columns."""
    uc = (nu - 1) / 2.0 + off_u / du
    return float(max(abs(np.arctan(-uc * du / sdd)), abs(np.arctan((nu - 1 - uc) * du / sdd))))


def short_scan(n_views: int, nu: int, nv: int, du: float, dv: float, nx: int, ny: int, nz: int,
               dx: float, overscan: float = 0.02, start: float = 0.0, **kw) -> Geometry:
    """A short scan: n_views uniform views from start to start + pi + 2 delta (both
    ends included), delta = the fan half-angle + overscan (rad)."""
    sdd = kw.get("sdd", 1500.0)
    delta = fan_half_angle(nu, du, sdd, kw.get("off_u", 0.0)) + overscan
    arc = np.pi + 2.0 * delta
    g = circular(n_views, nu, nv, du, dv, nx, ny, nz, dx, arc=arc * n_views / (n_views - 1), start=start, **kw)
    return g.with_(short_scan=True)


def gups(geom_or_updates, seconds: float) -> float:
    """Giga-updates per second, GUPS = Nx*Ny*Nz*Np / (T * 2^30) (Sec. 2.3)."""
    upd = geom_or_updates.updates if isinstance(geom_or_updates, Geometry) else int(geom_or_updates)
    return upd / (seconds * 2.0 ** 30)
