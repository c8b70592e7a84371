"""ctypes binding of the ifdk C-ABI (``include/ifdk.h``).

Argument marshalling only: every step of the reconstruction runs in the CUDA
library.  The functions keep the C names (``ifdk_create``, ``ifdk_filter``,
``ifdk_backproject``, ``ifdk_project`` ...); they accept torch CUDA tensors
(or raw device addresses) and enqueue on the current torch stream unless a
stream is given.  If the library is not built this module raises on first use:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from .geometry import Geometry

_LIBDIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib")
# IFDK_LIB_PATH selects another build of the same C-ABI (the checked build in tests)
LIB_PATH = os.environ.get("IFDK_LIB_PATH") or os.path.join(_LIBDIR, "libifdk.so")

IFDK_F32, IFDK_F16, IFDK_BF16 = 0, 1, 2
_ELEM = {0: 4, 1: 2, 2: 2}   # bytes per element of each storage type
IFDK_OK = 0
IFDK_ERR_INVALID, IFDK_ERR_GEOMETRY, IFDK_ERR_ALIGNMENT, IFDK_ERR_CUDA = -1, -2, -3, -4
IFDK_ERR_TIMEOUT, IFDK_ERR_NOMEM, IFDK_ERR_UNSUPPORTED, IFDK_ERR_BOUNDS = -5, -6, -7, -8

# every symbol include/ifdk.h declares
EXPORTS = ("ifdk_create", "ifdk_destroy", "ifdk_filter", "ifdk_filter_workspace_size", "ifdk_filter_noalloc",
           "ifdk_filter_adjoint",
           "ifdk_backproject", "ifdk_backproject_views", "ifdk_backproject_host",
           "ifdk_project", "ifdk_last_device_status", "ifdk_set_wait_limit", "ifdk_wait_selftest",
           "ifdk_backproject_info", "ifdk_query_backproject", "ifdk_query_rows", "ifdk_status_string",
           "ifdk_packed_size", "ifdk_pack_views", "ifdk_backproject_packed", "ifdk_set_view_pairing",
           "ifdk_backproject_packed_info", "ifdk_query_packed", "ifdk_volume_slices",
           "ifdk_set_view_split", "ifdk_view_split", "ifdk_filter_max", "ifdk_set_short_scan",
           "ifdk_backproject_packed_pairs", "ifdk_filter_views", "ifdk_backproject_packed_batch",
           "ifdk_arith_rate", "ifdk_iter_ratio", "ifdk_iter_update", "ifdk_set_test_abort",
           "ifdk_backproject_packed_quads")


class IfdkError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


class _GeometryC(ctypes.Structure):
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


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libifdk.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"ifdk CUDA library not built ({path}); run "
                               "paper_1909_02724_gb300.build.build() -- there is no CPU fallback")
        lib = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.ifdk_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_GeometryC)]
        lib.ifdk_destroy.argtypes = [vp]
        lib.ifdk_filter.argtypes = [vp, vp, vp, i32, i32, vp, ctypes.c_size_t, vp]
        lib.ifdk_filter_max.argtypes = [vp, vp, vp, i32, i32, vp, ctypes.c_size_t, vp, vp]
        lib.ifdk_filter_workspace_size.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_size_t),
                                                   ctypes.POINTER(ctypes.c_size_t)]
        lib.ifdk_filter_noalloc.argtypes = [vp, vp, vp, i32, i32, vp]
        lib.ifdk_filter_adjoint.argtypes = [vp, vp, vp, vp]
        lib.ifdk_backproject.argtypes = [vp, vp, i32, i32, i32, vp, vp]
        lib.ifdk_backproject_views.argtypes = [vp, vp, i32, i32, i32, vp, vp]
        lib.ifdk_backproject_host.argtypes = [vp, vp, i32, i32, i32, i32, i32, i32, vp, ctypes.c_size_t, vp, vp]
        lib.ifdk_query_rows.argtypes = [ctypes.POINTER(_GeometryC), i32, i32, ctypes.POINTER(i32),
                                        ctypes.POINTER(i32)]
        lib.ifdk_project.argtypes = [vp, vp, vp, i32, i32, vp]
        lib.ifdk_last_device_status.argtypes = [vp, vp]
        lib.ifdk_set_wait_limit.argtypes = [vp, ctypes.c_uint64]
        lib.ifdk_wait_selftest.argtypes = [vp, ctypes.c_uint64, vp]
        lib.ifdk_backproject_info.argtypes = [vp, i32, ctypes.POINTER(i64)]
        lib.ifdk_query_backproject.argtypes = [ctypes.POINTER(_GeometryC), i32, ctypes.POINTER(i64)]
        lib.ifdk_packed_size.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(i32),
                                         ctypes.POINTER(i32)]
        lib.ifdk_pack_views.argtypes = [vp, vp, i32, i32, vp, vp]
        lib.ifdk_backproject_packed.argtypes = [vp, vp, i32, i32, i32, vp, vp]
        lib.ifdk_set_view_pairing.argtypes = [vp, i32]
        lib.ifdk_backproject_packed_info.argtypes = [vp, i32, ctypes.POINTER(i64)]
        lib.ifdk_query_packed.argtypes = [ctypes.POINTER(_GeometryC), i32, i32, ctypes.POINTER(i64)]
        lib.ifdk_volume_slices.argtypes = [vp, vp, vp, i32, i32, i32, vp]
        lib.ifdk_set_view_split.argtypes = [vp, i32]
        lib.ifdk_set_short_scan.argtypes = [vp, i32]
        lib.ifdk_backproject_packed_pairs.argtypes = [vp, vp, i32, i32, i32, i32, i32, vp, vp]
        lib.ifdk_view_split.argtypes = [vp, i32, ctypes.POINTER(i32)]
        lib.ifdk_filter_views.argtypes = [vp, vp, vp, i32, i32, i32, i32, vp, ctypes.c_size_t, vp]
        lib.ifdk_backproject_packed_batch.argtypes = [vp, vp, i32, i32, i32, vp, vp]
        lib.ifdk_backproject_packed_quads.argtypes = [vp, vp, i32, i32, i32, vp, vp]
        lib.ifdk_set_test_abort.argtypes = [vp, i32]
        lib.ifdk_iter_ratio.argtypes = [vp, i32, vp, vp, vp, vp, i32, vp]
        lib.ifdk_iter_update.argtypes = [vp, i32, vp, vp, vp, ctypes.c_float, i32, vp]
        lib.ifdk_arith_rate.argtypes = [i32, i32, ctypes.c_longlong, vp, vp, ctypes.POINTER(i64), vp]
        lib.ifdk_status_string.argtypes = [i32]
        lib.ifdk_status_string.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name != "ifdk_status_string":
                getattr(lib, name).restype = i32
        _lib = lib
        return lib


def status_string(code: int) -> str:
    return load_library().ifdk_status_string(int(code)).decode()


def _check(rc: int, what: str) -> None:
    if rc != IFDK_OK:
        raise IfdkError(rc, what)


def _addr(x) -> int | None:
    """Device address of a torch tensor (or an int address / None)."""
    if x is None or isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def dtype_code(t) -> int:
    import torch
    m = {torch.float32: IFDK_F32, torch.float16: IFDK_F16, torch.bfloat16: IFDK_BF16}
    if t not in m:
        raise TypeError(f"unsupported projection storage type {t}")
    return m[t]


class _GeomHolder:
    def __init__(self, g: Geometry):
        import numpy as np
        self.angles = np.ascontiguousarray(g.angles, dtype=np.float64)
        self.weights = None if g.view_weights is None else np.ascontiguousarray(g.view_weights, dtype=np.float64)
        P = ctypes.POINTER(ctypes.c_double)
        self.c = _GeometryC(
            float(g.sid), float(g.sdd), int(g.nu), int(g.nv), float(g.du), float(g.dv),
            float(g.off_u), float(g.off_v), int(self.angles.shape[0]), self.angles.ctypes.data_as(P),
            None if self.weights is None else self.weights.ctypes.data_as(P),
            int(g.nx), int(g.ny), int(g.nz), float(g.dx), float(g.dy), float(g.dz), float(g.vol_off_z))


def ifdk_create(geom: Geometry) -> int:
    lib = load_library()
    h = _GeomHolder(geom)
    out = ctypes.c_void_p()
    _check(lib.ifdk_create(ctypes.byref(out), ctypes.byref(h.c)), "ifdk_create")
    return int(out.value)


def ifdk_destroy(plan: int) -> None:
    _check(load_library().ifdk_destroy(plan), "ifdk_destroy")


def ifdk_filter(plan: int, E, Q, q_dtype: int, split_terms: int, workspace=None, workspace_bytes: int = 0,
                stream=None) -> None:
    _check(load_library().ifdk_filter(plan, _addr(E), _addr(Q), int(q_dtype), int(split_terms), _addr(workspace),
                                      int(workspace_bytes), _stream(stream)), "ifdk_filter")


def ifdk_filter_max(plan: int, E, Q, q_dtype: int, split_terms: int, workspace, workspace_bytes: int, view_max,
                    stream=None) -> None:
    _check(load_library().ifdk_filter_max(plan, _addr(E), _addr(Q), int(q_dtype), int(split_terms),
                                          _addr(workspace), int(workspace_bytes), _addr(view_max), _stream(stream)),
           "ifdk_filter_max")


def ifdk_filter_workspace_size(plan: int, split_terms: int) -> tuple[int, int]:
    mn, pref = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load_library().ifdk_filter_workspace_size(plan, int(split_terms), ctypes.byref(mn), ctypes.byref(pref)),
           "ifdk_filter_workspace_size")
    return int(mn.value), int(pref.value)


def ifdk_filter_noalloc(plan: int, E, Q, q_dtype: int, split_terms: int, stream=None) -> None:
    """ifdk_filter's tensor-core path with the library's fixed 16 MiB workspace (allocates nothing)."""
    _check(load_library().ifdk_filter_noalloc(plan, _addr(E), _addr(Q), int(q_dtype), int(split_terms),
                                              _stream(stream)), "ifdk_filter_noalloc")


def ifdk_filter_adjoint(plan: int, G_Q, G_E, stream=None) -> None:
    _check(load_library().ifdk_filter_adjoint(plan, _addr(G_Q), _addr(G_E), _stream(stream)),
           "ifdk_filter_adjoint")


def ifdk_backproject(plan: int, Q, q_dtype: int, view_begin: int, view_count: int, vol, stream=None) -> None:
    _check(load_library().ifdk_backproject(plan, _addr(Q), int(q_dtype), int(view_begin), int(view_count),
                                           _addr(vol), _stream(stream)), "ifdk_backproject")


def ifdk_backproject_views(plan: int, Qv, q_dtype: int, view_begin: int, view_count: int, vol,
                           stream=None) -> None:
    """Qv holds only views [view_begin, view_begin + view_count)."""
    _check(load_library().ifdk_backproject_views(plan, _addr(Qv), int(q_dtype), int(view_begin), int(view_count),
                                                 _addr(vol), _stream(stream)), "ifdk_backproject_views")


def ifdk_backproject_host(plan: int, Q_host, q_dtype: int, host_nv: int, host_row0: int, view_begin: int,
                          view_count: int, chunk_views: int, staging, staging_bytes: int, vol, stream=None) -> None:
    """Q_host: host address (or CPU tensor) of [np][host_nv][nu]; staging: device buffer."""
    _check(load_library().ifdk_backproject_host(plan, _addr(Q_host), int(q_dtype), int(host_nv), int(host_row0),
                                                int(view_begin), int(view_count), int(chunk_views), _addr(staging),
                                                int(staging_bytes), _addr(vol), _stream(stream)),
           "ifdk_backproject_host")


def ifdk_query_rows(geom: Geometry, view_begin: int = 0, view_count: int | None = None) -> tuple[int, int]:
    """Host-only: (row_begin, row_count) of the detector rows the volume reads."""
    h = _GeomHolder(geom)
    r0, n = ctypes.c_int32(), ctypes.c_int32()
    vc = geom.np - view_begin if view_count is None else view_count
    _check(load_library().ifdk_query_rows(ctypes.byref(h.c), int(view_begin), int(vc), ctypes.byref(r0),
                                          ctypes.byref(n)), "ifdk_query_rows")
    return int(r0.value), int(n.value)


def ifdk_packed_size(plan: int, q_dtype: int) -> tuple[int, int, int]:
    """(bytes of one packed view, packed rows, elements per packed row)."""
    vb, rows, re = ctypes.c_size_t(), ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().ifdk_packed_size(plan, int(q_dtype), ctypes.byref(vb), ctypes.byref(rows), ctypes.byref(re)),
           "ifdk_packed_size")
    return int(vb.value), int(rows.value), int(re.value)


def ifdk_pack_views(plan: int, Q, q_dtype: int, view_count: int, Qp, stream=None) -> None:
    _check(load_library().ifdk_pack_views(plan, _addr(Q), int(q_dtype), int(view_count), _addr(Qp), _stream(stream)),
           "ifdk_pack_views")


def ifdk_backproject_packed(plan: int, Qp, q_dtype: int, view_begin: int, view_count: int, vol,
                            stream=None) -> None:
    _check(load_library().ifdk_backproject_packed(plan, _addr(Qp), int(q_dtype), int(view_begin), int(view_count),
                                                  _addr(vol), _stream(stream)), "ifdk_backproject_packed")


def ifdk_backproject_packed_pairs(plan: int, Qp, q_dtype: int, view_begin: int, view_count: int, pair_begin: int,
                                  pair_count: int, vol, stream=None) -> None:
    _check(load_library().ifdk_backproject_packed_pairs(plan, _addr(Qp), int(q_dtype), int(view_begin),
                                                        int(view_count), int(pair_begin), int(pair_count),
                                                        _addr(vol), _stream(stream)),
           "ifdk_backproject_packed_pairs")


def ifdk_filter_views(plan: int, Ev, Qv, q_dtype: int, split_terms: int, view_begin: int, view_count: int,
                      workspace=None, workspace_bytes: int = 0, stream=None) -> None:
    """Ev, Qv hold only views [view_begin, view_begin + view_count)."""
    _check(load_library().ifdk_filter_views(plan, _addr(Ev), _addr(Qv), int(q_dtype), int(split_terms),
                                            int(view_begin), int(view_count), _addr(workspace),
                                            int(workspace_bytes), _stream(stream)), "ifdk_filter_views")


def ifdk_backproject_packed_batch(plan: int, Qpb, q_dtype: int, view_begin: int, view_count: int, vol,
                                  stream=None) -> None:
    """Qpb: packed views [view_begin, +view_count) then their half-turn partners."""
    _check(load_library().ifdk_backproject_packed_batch(plan, _addr(Qpb), int(q_dtype), int(view_begin),
                                                        int(view_count), _addr(vol), _stream(stream)),
           "ifdk_backproject_packed_batch")


IFDK_SART, IFDK_MLEM = 0, 1


def ifdk_iter_ratio(plan: int, method: int, Pm, Ax, R, out, view_count: int, stream=None) -> None:
    """SART / MLEM ray-space ratio over view_count views (pointers at the range's first view)."""
    _check(load_library().ifdk_iter_ratio(plan, int(method), _addr(Pm), _addr(Ax), _addr(R), _addr(out),
                                          int(view_count), _stream(stream)), "ifdk_iter_ratio")


def ifdk_iter_update(plan: int, method: int, x, U, C, lam: float, nonneg: bool, stream=None) -> None:
    """SART / MLEM volume update x <- ..., U cleared."""
    _check(load_library().ifdk_iter_update(plan, int(method), _addr(x), _addr(U), _addr(C), float(lam),
                                           int(bool(nonneg)), _stream(stream)), "ifdk_iter_update")


def ifdk_backproject_packed_quads(plan: int, Qpq, q_dtype: int, view_begin: int, view_count: int, vol,
                                  stream=None) -> None:
    """Qpq: packed views [view_begin, +view_count) and the same shifted by np/4, np/2, 3np/4."""
    _check(load_library().ifdk_backproject_packed_quads(plan, _addr(Qpq), int(q_dtype), int(view_begin),
                                                        int(view_count), _addr(vol), _stream(stream)),
           "ifdk_backproject_packed_quads")


def ifdk_arith_rate(kind: int, blocks: int, iters: int, sink, clocks, stream=None) -> tuple[int, int]:
    """Launches the arithmetic rate probe; returns (instructions per thread, lanes per instruction)."""
    out = (ctypes.c_int64 * 2)()
    _check(load_library().ifdk_arith_rate(int(kind), int(blocks), int(iters), _addr(sink), _addr(clocks), out,
                                          _stream(stream)), "ifdk_arith_rate")
    return int(out[0]), int(out[1])


def pair_slab_depth(nz: int, pair_begin: int, pair_count: int) -> int:
    """nz_out of a pair-range volume: 2 pair_count, less the middle slice of an odd
    nz (its own mirror) when the range holds it."""
    npairs = (nz + 1) // 2
    return 2 * pair_count - (1 if nz % 2 and pair_begin + pair_count == npairs and pair_count > 0 else 0)


def _pairing_mode(mode) -> int:
    """False / True / 0 / 1 / 2 -> the C mode (0 off, 1 half-turn pairs, 2 quarter-turn quads)."""
    if isinstance(mode, bool):
        return 1 if mode else 0
    if mode not in (0, 1, 2):
        raise ValueError("view pairing mode must be 0, 1 or 2")
    return int(mode)


def ifdk_set_view_pairing(plan: int, enable) -> None:
    _check(load_library().ifdk_set_view_pairing(plan, _pairing_mode(enable)), "ifdk_set_view_pairing")


_PACKED_KEYS = ("path", "box_w", "box_h", "z_per_thread", "stages", "smem_bytes", "blocks", "fold_w", "align",
                "rows", "row_elems", "row0")


def ifdk_backproject_packed_info(plan: int, q_dtype: int) -> dict:
    arr = (ctypes.c_int64 * 12)()
    _check(load_library().ifdk_backproject_packed_info(plan, int(q_dtype), arr), "ifdk_backproject_packed_info")
    return dict(zip(_PACKED_KEYS, (int(v) for v in arr)))


def ifdk_query_packed(geom: Geometry, q_dtype: int, view_pairing=True) -> dict:
    """Host-only: the packed launch ifdk_backproject_packed would choose (view_pairing:
    False / True, or the mode 0, 1, 2 of ifdk_set_view_pairing)."""
    h = _GeomHolder(geom)
    arr = (ctypes.c_int64 * 12)()
    _check(load_library().ifdk_query_packed(ctypes.byref(h.c), int(q_dtype), _pairing_mode(view_pairing), arr),
           "ifdk_query_packed")
    return dict(zip(_PACKED_KEYS, (int(v) for v in arr)))


def ifdk_project(plan: int, vol, P, view_begin: int, view_count: int, stream=None) -> None:
    _check(load_library().ifdk_project(plan, _addr(vol), _addr(P), int(view_begin), int(view_count),
                                       _stream(stream)), "ifdk_project")


def ifdk_volume_slices(plan: int, vol, out, out_dtype: int, k_begin: int, k_count: int, stream=None) -> None:
    _check(load_library().ifdk_volume_slices(plan, _addr(vol), _addr(out), int(out_dtype), int(k_begin),
                                             int(k_count), _stream(stream)), "ifdk_volume_slices")


def ifdk_set_short_scan(plan: int, enable: bool) -> None:
    _check(load_library().ifdk_set_short_scan(plan, 1 if enable else 0), "ifdk_set_short_scan")


def ifdk_set_view_split(plan: int, max_splits: int) -> None:
    _check(load_library().ifdk_set_view_split(plan, int(max_splits)), "ifdk_set_view_split")


def ifdk_view_split(plan: int, q_dtype: int) -> int:
    out = ctypes.c_int(0)
    _check(load_library().ifdk_view_split(plan, int(q_dtype), ctypes.byref(out)), "ifdk_view_split")
    return int(out.value)


def ifdk_last_device_status(plan: int, stream=None) -> int:
    return int(load_library().ifdk_last_device_status(plan, _stream(stream)))


def ifdk_set_wait_limit(plan: int, nanoseconds: int) -> None:
    _check(load_library().ifdk_set_wait_limit(plan, int(nanoseconds)), "ifdk_set_wait_limit")


def ifdk_set_test_abort(plan: int, group: int) -> None:
    """Test hook: packed back-projections act as if the wait for view group `group` ran out (-1: off)."""
    _check(load_library().ifdk_set_test_abort(plan, int(group)), "ifdk_set_test_abort")


def ifdk_wait_selftest(plan: int, nanoseconds: int, stream=None) -> None:
    _check(load_library().ifdk_wait_selftest(plan, int(nanoseconds), _stream(stream)), "ifdk_wait_selftest")


def ifdk_backproject_info(plan: int, q_dtype: int) -> dict:
    arr = (ctypes.c_int64 * 8)()
    _check(load_library().ifdk_backproject_info(plan, int(q_dtype), arr), "ifdk_backproject_info")
    keys = ("path", "box_w", "box_h", "z_per_thread", "views_per_chunk", "smem_bytes", "blocks",
            "views_per_launch")
    return dict(zip(keys, (int(v) for v in arr)))


def ifdk_query_backproject(geom: Geometry, q_dtype: int) -> dict:
    """Host-only: the launch ifdk_backproject would choose (no device needed)."""
    h = _GeomHolder(geom)
    arr = (ctypes.c_int64 * 10)()
    _check(load_library().ifdk_query_backproject(ctypes.byref(h.c), int(q_dtype), arr),
           "ifdk_query_backproject")
    keys = ("path", "box_w", "box_h", "z_per_thread", "views_per_chunk", "smem_bytes", "blocks",
            "views_per_launch", "fold_w", "align")
    return dict(zip(keys, (int(v) for v in arr)))


class Plan:
    """Owns an ifdk plan for one geometry; methods take torch CUDA tensors."""

    def __init__(self, geom: Geometry):
        self.geom = geom
        self._ws = {}
        self.handle = ifdk_create(geom)
        if getattr(geom, "short_scan", False):
            try:
                ifdk_set_short_scan(self.handle, True)
            except Exception:
                self.close()
                raise

    def close(self) -> None:
        if self.handle:
            ifdk_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_views(self, t, name):
        g = self.geom
        if not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != (g.np, g.nv, g.nu):
            raise ValueError(f"{name} must be a contiguous CUDA tensor of shape {(g.np, g.nv, g.nu)}")

    def _check_vol(self, t):
        import torch
        g = self.geom
        if (not t.is_cuda or not t.is_contiguous() or t.dtype != torch.float32
                or tuple(t.shape) != (g.nx, g.ny, g.nz)):
            raise ValueError(f"vol must be a contiguous float32 CUDA tensor of shape {(g.nx, g.ny, g.nz)}")

    def workspace(self, split_terms: int, device):
        """Filter workspace (cached per plan and split count; caller-side allocation)."""
        import torch
        if split_terms == 0:
            return None, 0
        key = (split_terms, str(device))
        ws = self._ws.get(key)
        if ws is None:
            _, pref = ifdk_filter_workspace_size(self.handle, split_terms)
            ws = torch.empty(pref // 2 + 64, dtype=torch.bfloat16, device=device)
            self._ws[key] = ws
        base = ws.data_ptr()
        off = (-base) % 128
        return base + off, ws.numel() * 2 - off

    def filter(self, E, Q=None, dtype=None, split_terms: int | None = None, stream=None, view_max=None):
        """Algorithm 1 on the tensor cores: split_terms defaults to 3 BF16 terms
        for FP32 output and 2 for FP16 / BF16 output; 0 selects the SIMT kernel.
        view_max (optional): float32 CUDA tensor [np] that receives max |Q| per view
        in FP32 before the cast (ifdk_filter_max, the 16-bit range check)."""
        import torch
        self._check_views(E, "E")
        if E.dtype != torch.float32:
            raise ValueError("E must be float32")
        if Q is None:
            Q = torch.empty_like(E, dtype=dtype or torch.float32)
        self._check_views(Q, "Q")
        if split_terms is None:
            split_terms = 3 if Q.dtype == torch.float32 else 2
        ws, ws_bytes = self.workspace(split_terms, E.device)
        if view_max is None:
            ifdk_filter(self.handle, E, Q, dtype_code(Q.dtype), split_terms, ws, ws_bytes, stream)
        else:
            if (not view_max.is_cuda or view_max.dtype != torch.float32 or not view_max.is_contiguous()
                    or view_max.numel() != self.geom.np):
                raise ValueError(f"view_max must be a contiguous float32 CUDA tensor of {self.geom.np} elements")
            ifdk_filter_max(self.handle, E, Q, dtype_code(Q.dtype), split_terms, ws, ws_bytes, view_max, stream)
        return Q

    def filter_views(self, Ev, Qv=None, view_begin: int = 0, dtype=None, split_terms: int | None = None,
                     stream=None):
        """ifdk_filter_views: Ev (views, nv, nu) FP32 holds views [view_begin, view_begin + len(Ev));
        Qv receives them filtered (split_terms as in filter)."""
        import torch
        g = self.geom
        if (not Ev.is_cuda or not Ev.is_contiguous() or Ev.dim() != 3 or tuple(Ev.shape[1:]) != (g.nv, g.nu)
                or Ev.dtype != torch.float32):
            raise ValueError(f"Ev must be a contiguous float32 CUDA tensor of shape (views, {g.nv}, {g.nu})")
        if Qv is None:
            Qv = torch.empty_like(Ev, dtype=dtype or torch.float32)
        if not Qv.is_cuda or not Qv.is_contiguous() or tuple(Qv.shape) != tuple(Ev.shape):
            raise ValueError(f"Qv must be a contiguous CUDA tensor of shape {tuple(Ev.shape)}")
        if split_terms is None:
            split_terms = 3 if Qv.dtype == torch.float32 else 2
        ws, ws_bytes = self.workspace(split_terms, Ev.device)
        ifdk_filter_views(self.handle, Ev, Qv, dtype_code(Qv.dtype), split_terms, view_begin, Ev.shape[0], ws,
                          ws_bytes, stream)
        return Qv

    def filter_adjoint(self, G_Q, out=None, stream=None):
        import torch
        self._check_views(G_Q, "G_Q")
        if out is None:
            out = torch.empty_like(G_Q)
        ifdk_filter_adjoint(self.handle, G_Q, out, stream)
        return out

    def backproject(self, Q, vol=None, view_begin: int = 0, view_count: int | None = None, stream=None):
        import torch
        self._check_views(Q, "Q")
        g = self.geom
        if vol is None:
            vol = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device=Q.device)
        self._check_vol(vol)
        n = g.np - view_begin if view_count is None else view_count
        ifdk_backproject(self.handle, Q, dtype_code(Q.dtype), view_begin, n, vol, stream)
        return vol

    def backproject_views(self, Qv, vol=None, view_begin: int = 0, stream=None):
        """Back-project a tensor that holds only views [view_begin, view_begin + len(Qv))."""
        import torch
        g = self.geom
        if (not Qv.is_cuda or not Qv.is_contiguous() or Qv.dim() != 3 or tuple(Qv.shape[1:]) != (g.nv, g.nu)):
            raise ValueError(f"Qv must be a contiguous CUDA tensor of shape (views, {g.nv}, {g.nu})")
        if vol is None:
            vol = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device=Qv.device)
        self._check_vol(vol)
        ifdk_backproject_views(self.handle, Qv, dtype_code(Qv.dtype), view_begin, Qv.shape[0], vol, stream)
        return vol

    def staging_elems(self, dtype, chunk_views: int, packed: bool = True) -> int:
        """Elements of Q_host's dtype the streaming call needs: the two copy halves,
        plus the two packed halves when the packed path is used."""
        g = self.geom
        n = 2 * chunk_views * g.nv * g.nu
        if packed:
            try:
                vb, _, _ = ifdk_packed_size(self.handle, dtype_code(dtype))
            except IfdkError:
                vb = 0
            n += 2 * chunk_views * vb // _ELEM[dtype_code(dtype)]
        return n

    def backproject_host(self, Q_host, vol, staging=None, chunk_views: int = 64, host_row0: int = 0,
                         view_begin: int = 0, view_count: int | None = None, stream=None, packed: bool = True):
        """Back-project views streamed from a (pinned) CPU tensor [np][host_nv][nu]
        whose rows [host_row0, host_row0 + nv) are this plan's detector.
        staging: device buffer of Q_host's dtype (allocated here if None) of
        staging_elems() elements for the packed path (packed=True, when the
        plan has packed views) or 2 * chunk_views * nv * nu for the direct path.
        Asynchronous on `stream`."""
        import torch
        g = self.geom
        if (Q_host.is_cuda or not Q_host.is_contiguous() or Q_host.dim() != 3
                or Q_host.shape[0] != g.np or Q_host.shape[2] != g.nu):
            raise ValueError(f"Q_host must be a contiguous CPU tensor of shape ({g.np}, host_nv, {g.nu})")
        self._check_vol(vol)
        n = self.staging_elems(Q_host.dtype, chunk_views, packed)
        if staging is None:
            staging = torch.empty(n, dtype=Q_host.dtype, device=vol.device)
        if staging.dtype != Q_host.dtype or staging.numel() < 2 * chunk_views * g.nv * g.nu or not staging.is_cuda:
            raise ValueError("staging must be a CUDA tensor of Q_host's dtype with >= 2 * chunk_views * nv * nu elements")
        vc = g.np - view_begin if view_count is None else view_count
        ifdk_backproject_host(self.handle, Q_host, dtype_code(Q_host.dtype), Q_host.shape[1], host_row0, view_begin,
                              vc, chunk_views, staging, staging.numel() * staging.element_size(), vol, stream)
        return vol

    def packed_shape(self, dtype):
        """Shape (np, rows, row_elems, 4) of the packed views for storage dtype."""
        _, rows, re = ifdk_packed_size(self.handle, dtype_code(dtype))
        return (self.geom.np, rows, re, 4)

    def pack(self, Q, Qp=None, stream=None):
        """Packed views of Q (ifdk_pack_views): element (r, c) = Q[r][c], Q[2vc-r][c], Q[r][c+1], Q[2vc-r][c+1]."""
        import torch
        if not Q.is_cuda or not Q.is_contiguous() or Q.dim() != 3 or tuple(Q.shape[1:]) != (self.geom.nv, self.geom.nu):
            raise ValueError(f"Q must be a contiguous CUDA tensor of shape (views, {self.geom.nv}, {self.geom.nu})")
        shape = (Q.shape[0],) + self.packed_shape(Q.dtype)[1:]
        if Qp is None:
            Qp = torch.empty(shape, dtype=Q.dtype, device=Q.device)
        if not Qp.is_cuda or not Qp.is_contiguous() or tuple(Qp.shape) != shape or Qp.dtype != Q.dtype:
            raise ValueError(f"Qp must be a contiguous CUDA tensor of shape {shape} and Q's dtype")
        ifdk_pack_views(self.handle, Q, dtype_code(Q.dtype), Q.shape[0], Qp, stream)
        return Qp

    def backproject_packed(self, Qp, vol=None, view_begin: int = 0, view_count: int | None = None, stream=None):
        """Back-projection from packed views of all np views (ifdk_backproject_packed)."""
        import torch
        g = self.geom
        if not Qp.is_cuda or not Qp.is_contiguous() or tuple(Qp.shape) != self.packed_shape(Qp.dtype):
            raise ValueError(f"Qp must be a contiguous CUDA tensor of shape {self.packed_shape(Qp.dtype)}")
        if vol is None:
            vol = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device=Qp.device)
        self._check_vol(vol)
        n = g.np - view_begin if view_count is None else view_count
        ifdk_backproject_packed(self.handle, Qp, dtype_code(Qp.dtype), view_begin, n, vol, stream)
        return vol

    def backproject_packed_pairs(self, Qp, pair_begin: int, pair_count: int, vol=None, view_begin: int = 0,
                                 view_count: int | None = None, stream=None):
        """Mirror pairs [pair_begin, pair_begin + pair_count) only (ifdk_backproject_packed_pairs):
        vol [nx][ny][nz_out] holds the direct slab, then its mirror."""
        import torch
        g = self.geom
        if not Qp.is_cuda or not Qp.is_contiguous() or tuple(Qp.shape) != self.packed_shape(Qp.dtype):
            raise ValueError(f"Qp must be a contiguous CUDA tensor of shape {self.packed_shape(Qp.dtype)}")
        nz_out = pair_slab_depth(g.nz, pair_begin, pair_count)
        if vol is None:
            vol = torch.zeros((g.nx, g.ny, nz_out), dtype=torch.float32, device=Qp.device)
        if (not vol.is_cuda or not vol.is_contiguous() or vol.dtype != torch.float32
                or tuple(vol.shape) != (g.nx, g.ny, nz_out)):
            raise ValueError(f"vol must be a contiguous float32 CUDA tensor of shape {(g.nx, g.ny, nz_out)}")
        n = g.np - view_begin if view_count is None else view_count
        ifdk_backproject_packed_pairs(self.handle, Qp, dtype_code(Qp.dtype), view_begin, n, pair_begin, pair_count,
                                      vol, stream)
        return vol

    def backproject_packed_batch(self, Qpb, view_begin: int, view_count: int, vol=None, stream=None):
        """ifdk_backproject_packed_batch: Qpb (2 view_count, rows, row_elems, 4) holds the packed
        views [view_begin, +view_count) then their partners [view_begin + np/2, ...)."""
        import torch
        g = self.geom
        shape = (2 * view_count,) + self.packed_shape(Qpb.dtype)[1:]
        if not Qpb.is_cuda or not Qpb.is_contiguous() or tuple(Qpb.shape) != shape:
            raise ValueError(f"Qpb must be a contiguous CUDA tensor of shape {shape}")
        if vol is None:
            vol = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device=Qpb.device)
        self._check_vol(vol)
        ifdk_backproject_packed_batch(self.handle, Qpb, dtype_code(Qpb.dtype), view_begin, view_count, vol, stream)
        return vol

    def set_view_pairing(self, enable) -> None:
        """View pairing of the packed back-projection: False / 0 off, True / 1 half-turn pairs
        (the default), 2 quarter-turn quads where they apply."""
        ifdk_set_view_pairing(self.handle, enable)

    def backproject_packed_quads(self, Qpq, view_begin: int, view_count: int, vol=None, stream=None):
        """ifdk_backproject_packed_quads: Qpq (4 view_count, rows, row_elems, 4) holds the packed views
        [view_begin, +view_count) and the same range shifted by np/4, np/2 and 3np/4."""
        import torch
        g = self.geom
        shape = (4 * view_count,) + self.packed_shape(Qpq.dtype)[1:]
        if not Qpq.is_cuda or not Qpq.is_contiguous() or tuple(Qpq.shape) != shape:
            raise ValueError(f"Qpq must be a contiguous CUDA tensor of shape {shape}")
        if vol is None:
            vol = torch.zeros((g.nx, g.ny, g.nz), dtype=torch.float32, device=Qpq.device)
        self._check_vol(vol)
        ifdk_backproject_packed_quads(self.handle, Qpq, dtype_code(Qpq.dtype), view_begin, view_count, vol, stream)
        return vol

    def packed_info(self, dtype) -> dict:
        return ifdk_backproject_packed_info(self.handle, dtype_code(dtype))

    def has_packed(self, dtype) -> bool:
        """Whether packed views (and ifdk_backproject_packed) serve this geometry."""
        return self.packed_info(dtype)["path"] > 0

    def project(self, vol, P=None, view_begin: int = 0, view_count: int | None = None, stream=None):
        import torch
        self._check_vol(vol)
        g = self.geom
        if P is None:
            P = torch.zeros((g.np, g.nv, g.nu), dtype=torch.float32, device=vol.device)
        self._check_views(P, "P")
        n = g.np - view_begin if view_count is None else view_count
        ifdk_project(self.handle, vol, P, view_begin, n, stream)
        return P

    def slices(self, vol, out=None, dtype=None, k_begin: int = 0, k_count: int | None = None, stream=None):
        """Slices [k_begin, k_begin + k_count) of the k-fastest volume, i-fastest:
        out[k - k_begin][j][i] = vol[i][j][k] (ifdk_volume_slices)."""
        import torch
        self._check_vol(vol)
        g = self.geom
        n = g.nz - k_begin if k_count is None else k_count
        if out is None:
            out = torch.empty((n, g.ny, g.nx), dtype=dtype or torch.float32, device=vol.device)
        if not out.is_cuda or not out.is_contiguous() or tuple(out.shape) != (n, g.ny, g.nx):
            raise ValueError(f"out must be a contiguous CUDA tensor of shape ({n}, {g.ny}, {g.nx})")
        ifdk_volume_slices(self.handle, vol, out, dtype_code(out.dtype), k_begin, n, stream)
        return out

    def set_view_split(self, max_splits: int) -> None:
        """Cap on the view split of the packed back-projection (0 automatic, 1 off)."""
        ifdk_set_view_split(self.handle, max_splits)

    def view_split(self, dtype) -> int:
        """Parts of the view range a packed back-projection of all views uses (1: none)."""
        return ifdk_view_split(self.handle, dtype_code(dtype))

    def device_status(self, stream=None) -> int:
        return ifdk_last_device_status(self.handle, stream)

    def info(self, dtype) -> dict:
        import torch
        code = dtype if isinstance(dtype, int) else dtype_code(dtype if dtype is not None else torch.float32)
        return ifdk_backproject_info(self.handle, code)


IFDK_RATE_FFMA, IFDK_RATE_FFMA2, IFDK_RATE_HFMA2, IFDK_RATE_FMA_F32_F16, IFDK_RATE_LOP3 = 0, 1, 2, 3, 4
IFDK_RATE_FMA_F32_BF16 = 5
RATE_KINDS = {"ffma": IFDK_RATE_FFMA, "ffma2": IFDK_RATE_FFMA2, "hfma2": IFDK_RATE_HFMA2,
              "fma_f32_f16": IFDK_RATE_FMA_F32_F16, "lop3": IFDK_RATE_LOP3,
              "fma_f32_bf16": IFDK_RATE_FMA_F32_BF16}


def arith_rates(device=None, iters: int = 2048, kinds=tuple(RATE_KINDS)) -> dict:
    """Per-SM arithmetic rates of the GPU (ifdk_arith_rate): for each kind,
    lane operations and warp instructions per SM clock (median over blocks,
    each block timed by its own SM clock), with the SM count."""
    import numpy as np
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(n_sm * 1024, dtype=torch.float32, device=dev)
    clk = torch.empty(3 * n_sm, dtype=torch.int64, device=dev)
    out = {"n_sm": n_sm}
    for name in kinds:
        ifdk_arith_rate(RATE_KINDS[name], n_sm, 64, sink, clk)          # warm
        per_thread, lanes = ifdk_arith_rate(RATE_KINDS[name], n_sm, iters, sink, clk)
        torch.cuda.synchronize(dev)
        c = clk.view(n_sm, 3).cpu().numpy()
        cyc = (c[:, 1] - c[:, 0]).astype(np.float64)
        lane_ops = 1024.0 * per_thread * lanes
        rates = lane_ops / cyc
        out[name] = {"lane_ops_per_clk_sm": float(np.median(rates)), "lanes_per_instr": lanes,
                     "warp_instr_per_clk_sm": float(np.median(rates)) / (32 * lanes),
                     "min": float(rates.min()), "max": float(rates.max()),
                     "sms_seen": int(len(np.unique(c[:, 2])))}
    return out
