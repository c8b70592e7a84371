"""FP64 CPU oracle of the FDK hot path (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / reference leg of ``bench.py``.  The library path
(``paper_1909_02724_gb300``) never imports this package, and this package
imports nothing from it: the two share no code.

The arithmetic lives in ``ifdk_oracle.c`` (plain C, FP64, built with
``-O2 -ffp-contract=off``, no fast-math); this module only builds it with gcc
and marshals numpy arrays.  Each function names the passage of the paper it
follows (Chen et al., SC'19, arXiv 1909.02724):

* ``projection_matrices`` -- Eq. 2 with the M0 / Mrot / M1 matrices of Sec. 3.2.1
* ``cosine_weight``, ``ramlak``, ``filter_rows`` -- Algorithm 1
* ``backproject``, ``backproject_voxels`` -- Algorithm 2 with Algorithm 3
* ``project`` -- the exact adjoint of ``backproject``
* ``volume_slices`` -- the output stage of Algorithm 4 (I <- reshape(I~)), in numpy
* ``sart``, ``mlem`` -- the iterative solvers the paper names as further users of
  its back-projector (Sec. 1 and Sec. 6: SART, Andersen & Kak 1984; MLEM, Shepp &
  Vardi 1982), in numpy on ``project`` (A) and ``backproject`` (A^T), with
  ordered view subsets (Hudson & Larkin 1994)
* ``parker_weight``, ``short_scan_weights`` -- short-scan redundancy weights
  (Parker, Med. Phys. 9, 1982; not in the paper), in numpy; ``filter_rows`` /
  ``filter_views`` apply them for geometries with ``short_scan`` set

Geometry is passed as any object with the attributes of
``paper_1909_02724_gb300.geometry.Geometry`` (read by attribute name only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ifdk_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ifdk_oracle.c into oracle/lib/liboracle.so with gcc."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-D_GNU_SOURCE", "-O2", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Geom(ctypes.Structure):
    _fields_ = [
        ("sid", ctypes.c_double), ("sdd", ctypes.c_double),
        ("nu", ctypes.c_int), ("nv", ctypes.c_int),
        ("du", ctypes.c_double), ("dv", ctypes.c_double),
        ("off_u", ctypes.c_double), ("off_v", ctypes.c_double),
        ("np", ctypes.c_int), ("angles", ctypes.POINTER(ctypes.c_double)),
        ("view_weights", ctypes.POINTER(ctypes.c_double)),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("vol_off_z", ctypes.c_double),
    ]


_P = ctypes.POINTER
_d = ctypes.c_double
_i64 = ctypes.c_int64


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            G = _P(_Geom)
            lib.orc_projection_matrix.argtypes = [G, ctypes.c_int, _P(_d)]
            lib.orc_view_weight.argtypes = [G, ctypes.c_int]
            lib.orc_view_weight.restype = _d
            lib.orc_cosine_weight.argtypes = [G, _P(_d)]
            lib.orc_ramlak.argtypes = [ctypes.c_int, _P(_d)]
            for f in (lib.orc_filter_rows_direct, lib.orc_filter_rows_fft):
                f.argtypes = [G, _P(_d), _P(ctypes.c_int), ctypes.c_int, _P(_d)]
            lib.orc_backproject.argtypes = [G, _P(_d), ctypes.c_int, ctypes.c_int, _P(_d), ctypes.c_int]
            lib.orc_backproject.restype = ctypes.c_int
            lib.orc_backproject_voxels.argtypes = [G, _P(_d), _P(_i64), _P(_i64), _i64, _P(_d),
                                                   ctypes.c_int]
            lib.orc_backproject_voxels.restype = ctypes.c_int
            lib.orc_rows_needed.argtypes = [G, _P(_i64), _i64, _P(ctypes.c_ubyte)]
            lib.orc_project.argtypes = [G, _P(_d), ctypes.c_int, ctypes.c_int, _P(_d), ctypes.c_int]
            lib.orc_project.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct=_d):
    return a.ctypes.data_as(_P(ct))


class _GeomHolder:
    """Keeps the numpy arrays alive for as long as the ctypes struct is used."""

    def __init__(self, geom):
        self.angles = np.ascontiguousarray(np.asarray(geom.angles, dtype=np.float64))
        w = getattr(geom, "view_weights", None)
        self.weights = None if w is None else np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        self.s = _Geom(
            float(geom.sid), float(geom.sdd), int(geom.nu), int(geom.nv), float(geom.du),
            float(geom.dv), float(geom.off_u), float(geom.off_v), int(len(self.angles)),
            _ptr(self.angles), None if self.weights is None else _ptr(self.weights),
            int(geom.nx), int(geom.ny), int(geom.nz), float(geom.dx), float(geom.dy),
            float(geom.dz), float(geom.vol_off_z))

    @property
    def ref(self):
        return ctypes.byref(self.s)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def projection_matrices(geom) -> np.ndarray:
    """P_s (np x 3 x 4), Eq. 2: first three rows of M1 . Mrot(beta_s) . M0."""
    lib, g = _load(), _GeomHolder(geom)
    out = np.empty((len(g.angles), 3, 4))
    for s in range(len(g.angles)):
        lib.orc_projection_matrix(g.ref, s, _ptr(out[s]))
    return out


def view_weights(geom) -> np.ndarray:
    """Angular weight dbeta_s of each view (the spacing rule, or the user's weights)."""
    lib, g = _load(), _GeomHolder(geom)
    return np.array([lib.orc_view_weight(g.ref, s) for s in range(len(g.angles))])


def cosine_weight(geom) -> np.ndarray:
    """F_cos (nv x nu), Table 1 / Algorithm 1: D / sqrt(D^2 + a^2 + b^2)."""
    lib, g = _load(), _GeomHolder(geom)
    out = np.empty((geom.nv, geom.nu))
    lib.orc_cosine_weight(g.ref, _ptr(out))
    return out


def ramlak(n: int) -> np.ndarray:
    """Ram-Lak taps h(m), m = -(n-1)..n-1 (index m + n - 1)."""
    out = np.empty(2 * n - 1)
    _load().orc_ramlak(int(n), _ptr(out))
    return out


def parker_weight(beta, gamma, delta):
    """Parker's weight of the ray (beta, gamma) of a scan over [0, pi + 2 delta]:
    sin^2(pi/4 beta / (delta - gamma)) up to beta = 2 delta - 2 gamma, 1 up to
    pi - 2 gamma, sin^2(pi/4 (pi + 2 delta - beta) / (delta + gamma)) to the end,
    0 outside the scan."""
    b, gm = np.broadcast_arrays(np.asarray(beta, np.float64), np.asarray(gamma, np.float64))
    w = np.zeros(b.shape)
    rise = (b >= 0) & (b < 2 * delta - 2 * gm)
    flat = (b >= 2 * delta - 2 * gm) & (b <= np.pi - 2 * gm)
    fall = (b > np.pi - 2 * gm) & (b <= np.pi + 2 * delta)
    w[rise] = np.sin(np.pi / 4 * b[rise] / (delta - gm[rise])) ** 2
    w[flat] = 1.0
    w[fall] = np.sin(np.pi / 4 * (np.pi + 2 * delta - b[fall]) / (delta + gm[fall])) ** 2
    return w


def short_scan_weights(geom) -> np.ndarray:
    """(np, nu) factors 2 w(beta_s - beta_0, gamma_u) of a short scan, gamma_u the fan
    angle atan((u - u_c) Du / D) of column u and delta = (scan range - pi) / 2.  The 2
    replaces the 1/2 that the full-scan FDK constant (Kak-Slaney) holds for the rays'
    double cover."""
    uc = (geom.nu - 1) / 2.0 + geom.off_u / geom.du
    gamma = np.arctan((np.arange(geom.nu) - uc) * geom.du / geom.sdd)
    beta = np.asarray(geom.angles, np.float64) - geom.angles[0]
    delta = 0.5 * (beta[-1] - np.pi)
    assert np.all(np.diff(beta) > 0) and delta > np.abs(gamma).max() and beta[-1] < 2 * np.pi
    return 2.0 * parker_weight(beta[:, None], gamma[None, :], delta)


def filter_rows(geom, E_rows: np.ndarray, rows_v: np.ndarray, method: str = "auto",
                rows_s: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """Algorithm 1 on selected rows: Q = F_ramp (x) (E . F_cos).

    E_rows: (R, nu) raw projection rows; rows_v: (R,) detector row index of each
    (selects the F_cos row).  method: 'direct', 'fft' or 'auto' (fft for nu >= 256).
    rows_s: (R,) view index of each row, needed for a short-scan geometry (its rows
    are weighted by short_scan_weights before the filter).  threads: host threads
    over rows (default: every core).
    """
    lib, g = _load(), _GeomHolder(geom)
    E_rows = np.ascontiguousarray(E_rows, dtype=np.float64).reshape(-1, geom.nu)
    if getattr(geom, "short_scan", False):
        assert rows_s is not None, "short-scan rows need their view indices"
        E_rows = np.ascontiguousarray(E_rows * short_scan_weights(geom)[np.asarray(rows_s)])
    rows_v = np.ascontiguousarray(rows_v, dtype=np.int32).reshape(-1)
    assert rows_v.shape[0] == E_rows.shape[0]
    Q = np.empty_like(E_rows)
    if method == "auto":
        method = "fft" if geom.nu >= 256 else "direct"
    fn = lib.orc_filter_rows_fft if method == "fft" else lib.orc_filter_rows_direct
    n = E_rows.shape[0]
    nth = min(threads or default_threads(), max(1, n // 64))
    if nth <= 1:
        fn(g.ref, _ptr(E_rows), _ptr(rows_v, ctypes.c_int), n, _ptr(Q))
        return Q
    bounds = np.linspace(0, n, nth + 1).astype(int)

    def work(a, b):
        fn(g.ref, _ptr(E_rows[a:b]), _ptr(rows_v[a:b], ctypes.c_int), b - a, _ptr(Q[a:b]))

    ts = [threading.Thread(target=work, args=(int(a), int(b))) for a, b in zip(bounds[:-1], bounds[1:])]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return Q


def filter_views(geom, E: np.ndarray, method: str = "auto") -> np.ndarray:
    """Algorithm 1 on whole views: E (np, nv, nu) -> Q (np, nv, nu)."""
    npv = E.shape[0]
    rows_v = np.tile(np.arange(geom.nv, dtype=np.int32), npv)
    rows_s = np.repeat(np.arange(npv), geom.nv)
    return filter_rows(geom, E.reshape(-1, geom.nu), rows_v, method, rows_s).reshape(E.shape)


def backproject(geom, Q: np.ndarray, view_begin: int = 0, view_count: int | None = None,
                vol: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """Algorithm 2 (+ Algorithm 3, FDK weight): vol[i][j][k] += sum_s w_s f^2 interp2(Q_s, u, v)."""
    lib, g = _load(), _GeomHolder(geom)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    assert Q.shape == (len(g.angles), geom.nv, geom.nu)
    if view_count is None:
        view_count = len(g.angles) - view_begin
    if vol is None:
        vol = np.zeros((geom.nx, geom.ny, geom.nz))
    assert vol.dtype == np.float64 and vol.flags.c_contiguous
    rc = lib.orc_backproject(g.ref, _ptr(Q), int(view_begin), int(view_count), _ptr(vol),
                             int(threads or default_threads()))
    assert rc == 0
    return vol


def backproject_voxels(geom, Q: np.ndarray, voxels: np.ndarray, rowmap: np.ndarray | None = None,
                       threads: int | None = None) -> np.ndarray:
    """Algorithm 2 at selected voxels (N x 3 int array of (i, j, k)), all views.

    Q: dense (np, nv, nu), or sparse rows (R, nu) addressed by rowmap (np, nv) (-1 = absent).
    """
    lib, g = _load(), _GeomHolder(geom)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    vox = np.ascontiguousarray(voxels, dtype=np.int64).reshape(-1, 3)
    out = np.empty(vox.shape[0])
    rm = None if rowmap is None else np.ascontiguousarray(rowmap, dtype=np.int64)
    rc = lib.orc_backproject_voxels(g.ref, _ptr(Q), None if rm is None else _ptr(rm, _i64),
                                    _ptr(vox, _i64), vox.shape[0], _ptr(out),
                                    int(threads or default_threads()))
    if rc != 0:
        raise RuntimeError("backproject_voxels: a needed detector row was not supplied")
    return out


def rows_needed(geom, voxels: np.ndarray) -> np.ndarray:
    """Boolean (np, nv) mask of the detector rows that the voxels' bilinear taps touch."""
    lib, g = _load(), _GeomHolder(geom)
    vox = np.ascontiguousarray(voxels, dtype=np.int64).reshape(-1, 3)
    need = np.zeros((len(g.angles), geom.nv), dtype=np.uint8)
    lib.orc_rows_needed(g.ref, _ptr(vox, _i64), vox.shape[0], _ptr(need, ctypes.c_ubyte))
    return need.astype(bool)


def project(geom, vol: np.ndarray, view_begin: int = 0, view_count: int | None = None,
            out: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """Exact adjoint of ``backproject``: weighted bilinear splat of the volume into the views."""
    lib, g = _load(), _GeomHolder(geom)
    vol = np.ascontiguousarray(vol, dtype=np.float64)
    assert vol.shape == (geom.nx, geom.ny, geom.nz)
    if view_count is None:
        view_count = len(g.angles) - view_begin
    if out is None:
        out = np.zeros((len(g.angles), geom.nv, geom.nu))
    lib.orc_project(g.ref, _ptr(vol), int(view_begin), int(view_count), _ptr(out),
                    int(threads or default_threads()))
    return out


def fdk(geom, E: np.ndarray, threads: int | None = None) -> np.ndarray:
    """Full FDK in FP64: Algorithm 1 then Algorithm 2."""
    return backproject(geom, filter_views(geom, np.asarray(E, dtype=np.float64)), threads=threads)


def round_bf16_bits(x: np.ndarray) -> np.ndarray:
    """bfloat16 bit patterns (uint16) of FP32 values, rounded to nearest, ties to
    even: the 32-bit pattern keeps its top 16 bits, plus one when the dropped low
    16 bits exceed half a unit, or equal it and the kept part is odd (finite
    values only)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    hi, lo = b >> 16, b & 0xFFFF
    up = (lo > 0x8000) | ((lo == 0x8000) & ((hi & 1) == 1))
    return (hi + up).astype(np.uint16)


def volume_slices(vol: np.ndarray, k_begin: int = 0, k_count: int | None = None,
                  dtype: str = "f32") -> np.ndarray:
    """Output stage of Algorithm 4, I <- reshape(I~): slices [k_begin, k_begin + k_count)
    of the k-fastest volume [nx][ny][nz] as an i-fastest [k_count][ny][nx] array,
    out[k - k_begin][j][i] = vol[i][j][k].  dtype "f32" keeps the FP32 values, "f16"
    rounds to nearest even (numpy float16), "bf16" returns round_bf16_bits."""
    vol = np.asarray(vol, dtype=np.float32)
    nz = vol.shape[2]
    if k_count is None:
        k_count = nz - k_begin
    if k_begin < 0 or k_count < 0 or k_begin + k_count > nz:
        raise ValueError("slice range outside the volume")
    out = np.ascontiguousarray(np.transpose(vol[:, :, k_begin:k_begin + k_count], (2, 1, 0)))
    if dtype == "f32":
        return out
    if dtype == "f16":
        with np.errstate(over="ignore"):      # beyond the largest half: infinity, as rounding gives
            return out.astype(np.float16)
    if dtype == "bf16":
        return round_bf16_bits(out)
    raise ValueError(dtype)


# --------------------------------------------------------------------------
# Iterative solvers on the back-projection / adjoint pair.  The system matrix
# is A = project (volume -> views, the exact adjoint of the back-projection)
# and A^T = backproject.  A subset is a list of (view_begin, view_count)
# ranges; an iteration visits the subsets in order.
# --------------------------------------------------------------------------

def _project_ranges(geom, x, ranges, threads=None):
    out = np.zeros((geom.np, geom.nv, geom.nu))
    for b, c in ranges:
        project(geom, x, b, c, out=out, threads=threads)
    return out


def _backproject_ranges(geom, q, ranges, threads=None):
    vol = np.zeros((geom.nx, geom.ny, geom.nz))
    for b, c in ranges:
        backproject(geom, q, b, c, vol=vol, threads=threads)
    return vol


def _views_of(ranges, np_):
    m = np.zeros(np_, dtype=bool)
    for b, c in ranges:
        m[b:b + c] = True
    return m


def column_sums(geom, ranges, threads=None) -> np.ndarray:
    """C_S = A_S^T 1: the back-projection of all-ones views over the subset's views."""
    return _backproject_ranges(geom, np.ones((geom.np, geom.nv, geom.nu)), ranges, threads)


def row_sums(geom, threads=None) -> np.ndarray:
    """R = A 1: the projection of an all-ones volume (every view)."""
    return project(geom, np.ones((geom.nx, geom.ny, geom.nz)), threads=threads)


def sart(geom, p: np.ndarray, x0: np.ndarray, iterations: int, subsets, lam: float = 1.0,
         nonneg: bool = False, threads=None) -> list:
    """SART (Andersen & Kak, Ultrasonic Imaging 6, 1984), block form over ordered
    view subsets: for each subset S in turn,
        x <- x + lam * (A_S^T ((p - A x) / R)) / C_S
    with R = A 1 (row sums over every voxel) and C_S = A_S^T 1 (column sums over
    the subset's rays); a ray with R = 0 contributes nothing, a voxel with
    C_S = 0 is left as it is; nonneg clips x at 0 after each update.  One
    subset holding every view is SIRT.  Returns the iterate after each
    iteration (a pass over all subsets)."""
    R = row_sums(geom, threads)
    Cs = [column_sums(geom, S, threads) for S in subsets]
    x = np.array(x0, dtype=np.float64, copy=True)
    out = []
    for _ in range(iterations):
        for S, C in zip(subsets, Cs):
            m = _views_of(S, geom.np)
            Ax = _project_ranges(geom, x, S, threads)
            r = np.zeros_like(Ax)
            np.divide(p - Ax, R, out=r, where=(R > 0) & m[:, None, None])
            U = _backproject_ranges(geom, r, S, threads)
            step = np.zeros_like(x)
            np.divide(U, C, out=step, where=C > 0)
            x = x + lam * step
            if nonneg:
                x = np.maximum(x, 0.0)
        out.append(x.copy())
    return out


def mlem(geom, p: np.ndarray, x0: np.ndarray, iterations: int, subsets, threads=None) -> list:
    """MLEM (Shepp & Vardi, IEEE TMI 1, 1982) over ordered view subsets (OS-EM,
    Hudson & Larkin, IEEE TMI 13, 1994): for each subset S in turn,
        x <- x * (A_S^T (p / A x)) / C_S
    with C_S = A_S^T 1; a ray with A x = 0 contributes nothing, a voxel with
    C_S = 0 is left as it is.  p >= 0, x0 > 0.  Returns the iterate after each
    iteration."""
    Cs = [column_sums(geom, S, threads) for S in subsets]
    x = np.array(x0, dtype=np.float64, copy=True)
    out = []
    for _ in range(iterations):
        for S, C in zip(subsets, Cs):
            m = _views_of(S, geom.np)
            Ax = _project_ranges(geom, x, S, threads)
            ratio = np.zeros_like(Ax)
            np.divide(p, Ax, out=ratio, where=(Ax > 0) & m[:, None, None])
            U = _backproject_ranges(geom, ratio, S, threads)
            upd = x * U
            x = np.where(C > 0, upd / np.where(C > 0, C, 1.0), x)
        out.append(x.copy())
    return out
