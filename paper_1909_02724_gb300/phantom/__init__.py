"""Seeded synthetic inputs: ellipsoid phantoms and their exact cone-beam line integrals.

This module is the input generator shared by the tests, the oracle checks and
the benchmark.  It holds none of the reconstruction arithmetic (no cosine
weight, no ramp filter, no back-projection): it only describes objects in
world coordinates and integrates them along the scanner's rays.

World frame (derived from the M0 / Mrot / M1 matrices of Eq. 2): the source of
view beta sits at (-d sin beta, -d cos beta, 0); detector pixel (iu, iv) sits at
R(beta)^T (a, D - d) in XY and Z = -b, with a = (iu - u_c) Du, b = (iv - v_c) Dv,
u_c = (Nu-1)/2 + off_u/Du, v_c = (Nv-1)/2 + off_v/Dv, R(beta) the rotation by +beta.

The paper's measurements use Shepp-Logan projections made by RTK's forward
projector (Sec. 5.1); RTK and those files are not available, so seeded
ellipsoid sets with the same structure (additive ellipsoids of densities
0.1..1 inside the field of view) stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from ..geometry import Geometry, circular


@dataclass
class Ellipsoids:
    centre: np.ndarray   # (N, 3) mm
    axes: np.ndarray     # (N, 3) semi-axes (mm)
    rot: np.ndarray      # (N, 3, 3) columns = ellipsoid axes in world coordinates
    rho: np.ndarray      # (N,) density (additive)

    def __len__(self):
        return int(self.rho.shape[0])

    def packed(self) -> np.ndarray:
        """(N, 16) float64 rows: centre(3), 1/axes(3), rot row-major(9), rho."""
        n = len(self)
        out = np.zeros((n, 16))
        out[:, 0:3] = self.centre
        out[:, 3:6] = 1.0 / self.axes
        out[:, 6:15] = self.rot.reshape(n, 9)
        out[:, 15] = self.rho
        return out

    def mirrored_z(self) -> "Ellipsoids":
        """The set together with its mirror image about the plane Z = 0."""
        flip = np.diag([1.0, 1.0, -1.0])
        c2 = self.centre * np.array([1.0, 1.0, -1.0])
        r2 = np.einsum("ab,nbc->nac", flip, self.rot)
        return Ellipsoids(np.concatenate([self.centre, c2]), np.concatenate([self.axes, self.axes]),
                          np.concatenate([self.rot, r2]), np.concatenate([self.rho, self.rho]))


def sphere(radius: float, rho: float = 1.0, centre=(0.0, 0.0, 0.0)) -> Ellipsoids:
    return Ellipsoids(np.array([centre], dtype=np.float64), np.full((1, 3), float(radius)),
                      np.eye(3)[None].copy(), np.array([float(rho)]))


def _quat_to_rot(q: np.ndarray) -> np.ndarray:
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def random_ellipsoids(n: int, r_safe: float, seed: int) -> Ellipsoids:
    """Seeded ellipsoid set: centres uniform in a ball of radius 0.5 r_safe,
    semi-axes uniform in [0.05, 0.45] r_safe, uniformly random orientation
    (normalised Gaussian quaternion), densities uniform in [0.1, 1.0]; every
    ellipsoid lies inside the sphere of radius 0.95 r_safe."""
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = 0.5 * r_safe * rng.uniform(size=n) ** (1.0 / 3.0)
    centre = d * r[:, None]
    axes = rng.uniform(0.05, 0.45, size=(n, 3)) * r_safe
    rot = _quat_to_rot(rng.normal(size=(n, 4)))
    rho = rng.uniform(0.1, 1.0, size=n)
    return Ellipsoids(centre, axes, rot, rho)


def principal_point(geom: Geometry) -> tuple[float, float]:
    return ((geom.nu - 1) / 2.0 + geom.off_u / geom.du, (geom.nv - 1) / 2.0 + geom.off_v / geom.dv)


def safe_radius(geom: Geometry) -> float:
    """Radius of a centred ball that every view sees untruncated (no ray of
    the ball leaves the detector), limited by the volume's own extent."""
    uc, vc = principal_point(geom)
    half_w = min(uc, geom.nu - 1 - uc) * geom.du
    half_h = min(vc, geom.nv - 1 - vc) * geom.dv
    r_fan = geom.sid * np.sin(np.arctan(half_w / geom.sdd))
    r_cone = half_h * geom.sid / (geom.sdd + half_h)
    r_vol = 0.5 * min(geom.nx * geom.dx, geom.ny * geom.dy, geom.nz * geom.dz)
    return float(min(r_fan, r_cone, r_vol))


def source_positions(geom: Geometry, views=None) -> np.ndarray:
    b = geom.angles if views is None else geom.angles[np.asarray(views)]
    return np.stack([-geom.sid * np.sin(b), -geom.sid * np.cos(b), np.zeros_like(b)], -1)


def pixel_positions(geom: Geometry, beta: float, iu: np.ndarray, iv: np.ndarray) -> np.ndarray:
    """World position of detector pixel centres (iu, iv) of the view at angle beta."""
    uc, vc = principal_point(geom)
    a = (np.asarray(iu, dtype=np.float64) - uc) * geom.du
    b = (np.asarray(iv, dtype=np.float64) - vc) * geom.dv
    a, b = np.broadcast_arrays(a, b)
    t = geom.sdd - geom.sid
    c, s = np.cos(beta), np.sin(beta)
    return np.stack([c * a + s * t, -s * a + c * t, -b], -1)


def chord_lengths(ell: Ellipsoids, src: np.ndarray, dst: np.ndarray) -> np.ndarray:
    """Sum over ellipsoids of rho * (length of the line src->dst inside it).

    src: (3,), dst: (..., 3).  The quadratic is set up about the point of the
    line nearest each centre so that it stays well conditioned."""
    d = dst - src
    d = d / np.linalg.norm(d, axis=-1, keepdims=True)
    total = np.zeros(d.shape[:-1])
    for e in range(len(ell)):
        c = ell.centre[e]
        t0 = np.einsum("...k,k->...", d, c - src)
        p0 = src + t0[..., None] * d
        m = ell.rot[e].T / ell.axes[e][:, None]          # diag(1/a) R^T
        sp = np.einsum("ij,...j->...i", m, p0 - c)
        dp = np.einsum("ij,...j->...i", m, d)
        A = np.einsum("...i,...i->...", dp, dp)
        B = np.einsum("...i,...i->...", sp, dp)
        C = np.einsum("...i,...i->...", sp, sp) - 1.0
        disc = B * B - A * C
        total += ell.rho[e] * np.where(disc > 0, 2.0 * np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)
    return total


def line_integrals(ell: Ellipsoids, geom: Geometry, views=None) -> np.ndarray:
    """E[s][iv][iu]: exact line integrals from the source to each pixel centre (FP64)."""
    views = np.arange(geom.np) if views is None else np.asarray(views)
    iv, iu = np.meshgrid(np.arange(geom.nv), np.arange(geom.nu), indexing="ij")
    out = np.empty((len(views), geom.nv, geom.nu))
    for n, s in enumerate(views):
        beta = geom.angles[s]
        src = np.array([-geom.sid * np.sin(beta), -geom.sid * np.cos(beta), 0.0])
        out[n] = chord_lengths(ell, src, pixel_positions(geom, beta, iu, iv))
    return out


def line_integral_rows(ell: Ellipsoids, geom: Geometry, s_idx: np.ndarray, r_idx: np.ndarray,
                       threads: int | None = None, chunk: int = 32) -> np.ndarray:
    """E[s_idx[n]][r_idx[n]][:] for selected detector rows (FP64): the same chords as
    line_integrals, for many views at once (rows in chunks over host threads)."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    s_idx, r_idx = np.asarray(s_idx), np.asarray(r_idx)
    out = np.empty((len(s_idx), geom.nu))
    iu = np.arange(geom.nu)

    def work(a):
        b = min(a + chunk, len(s_idx))
        for s in np.unique(s_idx[a:b]):
            sel = a + np.nonzero(s_idx[a:b] == s)[0]
            src = source_positions(geom, [s])[0]
            out[sel] = chord_lengths(ell, src, pixel_positions(geom, geom.angles[s], iu[None, :], r_idx[sel][:, None]))

    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        list(ex.map(work, range(0, len(s_idx), chunk)))
    return out


def add_noise(E: np.ndarray, rel_sigma: float, seed: int) -> np.ndarray:
    """Gaussian noise with sigma = rel_sigma * max(E), seeded."""
    rng = np.random.default_rng(seed)
    return E + rng.normal(scale=rel_sigma * float(E.max()), size=E.shape)


# --------------------------------------------------------------------------
# Workloads: the fixed geometry d = 1000 mm, D = 1500 mm, scaled by keeping a
# 64 mm volume and a 96 mm detector (about one detector pixel per voxel).
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    geom: Geometry
    n_ellipsoids: int
    seed: int
    noise: float = 0.0

    def phantom(self) -> Ellipsoids:
        return random_ellipsoids(self.n_ellipsoids, 0.9 * safe_radius(self.geom), self.seed)


def scaled_geometry(n_vol: int, n_det: int, n_views: int, nz: int | None = None,
                    n_det_v: int | None = None, fov: float = 64.0, det: float = 96.0) -> Geometry:
    nz = n_vol if nz is None else nz
    n_det_v = n_det if n_det_v is None else n_det_v
    return circular(n_views, n_det, n_det_v, det / n_det, det / n_det, n_vol, n_vol, nz,
                    fov / n_vol)


def workload(name: str) -> Workload:
    """Named workloads (seed 1909 + index):

    fdk64      64^3 from 64 views of 64x64 (1 mm voxels, 1.5 mm pixels), 10 ellipsoids
    fdk512     512^3 from 512 views of 512x512, 30 ellipsoids + 1% Gaussian noise
    fdk2048    2048^3 from 2048 views of 2048x2048, 100 ellipsoids
    grad256    256^3 from 360 views of 384x384, 20 ellipsoids
    grad32     32^3 from 48 views of 48x48 (finite-difference check), 20 ellipsoids
    slab4096   central 4096x4096x256 slab of a 4096^3 grid, 2048 views of 4096x4096, 200 ellipsoids
    """
    if name == "fdk64":
        return Workload(name, scaled_geometry(64, 64, 64), 10, 1909 + 0)
    if name == "fdk512":
        return Workload(name, scaled_geometry(512, 512, 512), 30, 1909 + 1, noise=0.01)
    if name == "fdk2048":
        return Workload(name, scaled_geometry(2048, 2048, 2048), 100, 1909 + 2)
    if name == "grad256":
        return Workload(name, scaled_geometry(256, 384, 360), 20, 1909 + 3)
    if name == "grad32":
        return Workload(name, scaled_geometry(32, 48, 48), 20, 1909 + 3)
    if name == "slab4096":
        g = scaled_geometry(4096, 4096, 2048, nz=256)
        return Workload(name, g, 200, 1909 + 4)
    raise KeyError(name)


# --------------------------------------------------------------------------
# FP32 CUDA generator (phantom.cu, its own shared library) for large workloads.
# --------------------------------------------------------------------------

_gpu_lib = None


def _load_gpu():
    global _gpu_lib
    if _gpu_lib is None:
        import ctypes
        import os
        path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "lib",
                            "libifdk_phantom.so")
        if not os.path.exists(path):
            raise RuntimeError(f"phantom generator library not built ({path})")
        lib = ctypes.CDLL(path)
        d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        lib.ifdk_phantom_project.argtypes = [vp, i, d, d, i, i, d, d, d, d, vp, i, i, vp, vp]
        lib.ifdk_phantom_project.restype = i
        _gpu_lib = lib
    return _gpu_lib


def line_integrals_gpu(ell: Ellipsoids, geom: Geometry, out=None, view_begin: int = 0,
                       view_count: int | None = None, chunk: int = 256):
    """E (torch float32 CUDA tensor [view_count][nv][nu]) from the FP32 CUDA generator."""
    import torch
    n = geom.np - view_begin if view_count is None else view_count
    if out is None:
        out = torch.empty((n, geom.nv, geom.nu), dtype=torch.float32, device="cuda")
    packed = np.ascontiguousarray(ell.packed())
    angles = np.ascontiguousarray(geom.angles)
    lib = _load_gpu()
    stream = torch.cuda.current_stream().cuda_stream
    for s0 in range(0, n, chunk):
        c = min(chunk, n - s0)
        rc = lib.ifdk_phantom_project(packed.ctypes.data, len(ell), geom.sid, geom.sdd, geom.nu, geom.nv,
                                      geom.du, geom.dv, geom.off_u, geom.off_v, angles.ctypes.data,
                                      view_begin + s0, c, out[s0:s0 + c].data_ptr(), stream)
        if rc != 0:
            raise RuntimeError(f"ifdk_phantom_project failed ({rc})")
    return out


def workload_projections_gpu(w: Workload, out=None):
    """Projections of a named workload on the GPU (seeded phantom, then seeded noise)."""
    import torch
    E = line_integrals_gpu(w.phantom(), w.geom, out=out)
    if w.noise:
        gen = torch.Generator(device=E.device)
        gen.manual_seed(w.seed)
        sigma = w.noise * float(E.max())
        E.add_(torch.randn(E.shape, generator=gen, device=E.device, dtype=E.dtype), alpha=sigma)
    return E
