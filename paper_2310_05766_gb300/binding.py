"""Thin Python binding of libtsdf_gb300.so (the C ABI in include/tsdf.h).

Argument marshalling only: every step of the TSDF path runs in the library's
CUDA kernels. PyTorch is used for device memory (tensors' data pointers) and
streams (`torch.cuda.current_stream().cuda_stream`). There is no CPU
fallback: if the library has not been built, loading it raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

TSDF_OK = 0
TSDF_ERR_INVALID = -1
TSDF_ERR_OOM = -2
TSDF_ERR_CUDA = -3
TSDF_ERR_TIMEOUT = -4
TSDF_ERR_ADMISSION = -5
TSDF_ERR_BUSY = -6
TSDF_ERR_IO = -7
TSDF_ERR_CAPACITY = -8
TSDF_ERR_DEGENERATE = -9
TSDF_REDUCE_WSUM = 0
TSDF_REDUCE_MIN_ABS = 1
TSDF_FLAG_STEP_VALUE = 1
TSDF_FLAG_SCAN_WEIGHT = 2
TSDF_MAX_POINTS = (1 << 22) - 1
TSDF_OPT_WARP_MERGE = 1
TSDF_OPT_STEPS_PER_THREAD = 2
TSDF_OPT_PDL = 3
TSDF_OPT_REDUCTION = 4
TSDF_OPT_SORT_CAPACITY = 5
TSDF_OPT_HOST_ZERO_COPY = 6
TSDF_REDUCTION_ATOMIC = 0
TSDF_REDUCTION_SORT = 1
TSDF_REDUCTION_POOL = 2
TSDF_REDUCTION_AUTO = 3
TSDF_OPT_POOL_BRICKS = 7
TSDF_OPT_STORE_DEVICE_CHUNKS = 8
TSDF_OPT_STORE_SPILL_AGE = 9
TSDF_OPT_LAUNCH_GRAPH = 10
TSDF_BATCH_OPT_GRAPH = 1
TSDF_BATCH_OPT_AUTOTUNE = 2
TSDF_BATCH_OPT_CONFIG = 3
TSDF_BATCH_OPT_SPIN_LIMIT = 4
TSDF_BATCH_OPT_TEST_MISSING_ARRIVALS = 5
TSDF_BATCH_OPT_GRID_FRACTION = 6
TSDF_BATCH_OPT_TUNE_SORT = 7
TSDF_BATCH_OPT_CTA_BRICK_CACHE = 8
TSDF_STATIC_MAX_VOXELS = 1 << 21
TSDF_STATIC_MAX_POINTS = 1 << 17


class TsdfError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {tsdf_error_string(code)} ({code})"
                         + (f", cudaError {tsdf_last_cuda_error()}" if code == TSDF_ERR_CUDA else ""))


class tsdf_params(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("voxel_size", ctypes.c_float), ("tau", ctypes.c_float),
                ("w_max", ctypes.c_int32), ("delta_z", ctypes.c_float), ("r_min", ctypes.c_float),
                ("r_max", ctypes.c_float), ("reduce", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("origin", ctypes.c_int64 * 3)]


class tsdf_scan_stats(ctypes.Structure):
    _fields_ = [("valid_rays", ctypes.c_int64), ("hits", ctypes.c_int64), ("touched", ctypes.c_int64)]


class tsdf_register_result(ctypes.Structure):
    _fields_ = [("used_points", ctypes.c_int64), ("rms", ctypes.c_double), ("step", ctypes.c_double),
                ("iterations", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class tsdf_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class tsdf_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_points", ctypes.c_int64), ("max_batch", ctypes.c_int32),
                ("streams", ctypes.c_int32), ("max_outstanding", ctypes.c_int32), ("store_chunks", ctypes.c_int32)]


class tsdf_request_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("session", ctypes.c_int32), ("status", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("reserved", ctypes.c_int32), ("stats", tsdf_scan_stats),
                ("t_submit_us", ctypes.c_double), ("t_start_us", ctypes.c_double), ("t_done_us", ctypes.c_double)]


class tsdf_server_stats(ctypes.Structure):
    _fields_ = [("sessions", ctypes.c_int32), ("reserved", ctypes.c_int32), ("used_bytes", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("batches", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("mean_batch", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the CUDA library. Raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: run __graft_entry__.build() "
                           "(the TSDF path has no CPU fallback)")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    f32p = P(ctypes.c_float)
    L.tsdf_map_create.argtypes = [P(tsdf_params), P(vp)]
    L.tsdf_map_destroy.argtypes = [vp]
    # the pose by address (the per-scan calls skip building a ctypes pointer)
    L.tsdf_integrate.argtypes = [vp, vp, i64, vp, vp]
    L.tsdf_integrate_host.argtypes = [vp, vp, i64, vp, vp]
    L.tsdf_shift.argtypes = [vp, P(i64), vp]
    L.tsdf_read.argtypes = [vp, P(i64), P(i64), vp, vp, vp]
    L.tsdf_write.argtypes = [vp, P(i64), P(i64), vp, vp, vp]
    L.tsdf_stats.argtypes = [vp, P(tsdf_scan_stats), vp]
    L.tsdf_get_origin.argtypes = [vp, P(i64)]
    L.tsdf_grid_device_ptr.argtypes = [vp, P(vp)]
    L.tsdf_set_option.argtypes = [vp, ctypes.c_int32, ctypes.c_int64]
    L.tsdf_profile_enable.argtypes = [vp, ctypes.c_int32]
    L.tsdf_profile_read.argtypes = [vp, P(tsdf_kernel_time), ctypes.c_int32, P(ctypes.c_int32)]
    L.tsdf_probe_reduction_rate.argtypes = [ctypes.c_int32, P(ctypes.c_double), vp]
    L.tsdf_map_save.argtypes = [vp, ctypes.c_char_p, vp]
    L.tsdf_map_device_bytes.argtypes = [vp, P(i64)]
    L.tsdf_map_reserve_store.argtypes = [vp, i64]
    L.tsdf_get_store_stats.argtypes = [vp, vp]
    L.tsdf_map_set_store_file.argtypes = [vp, ctypes.c_char_p, i64]
    L.tsdf_get_reduction.argtypes = [vp, P(ctypes.c_int32)]
    L.tsdf_extract_mesh.argtypes = [vp, ctypes.c_int32, vp, i64, P(i64), vp]
    L.tsdf_register_system.argtypes = [vp, vp, i64, f32p, ctypes.c_int32, P(ctypes.c_double), vp]
    L.tsdf_register.argtypes = [vp, vp, i64, f32p, ctypes.c_int32, ctypes.c_int32, P(tsdf_register_result), vp]
    L.tsdf_extract_surface.argtypes = [vp, ctypes.c_int32, vp, i64, P(i64), vp]
    L.tsdf_map_load.argtypes = [ctypes.c_char_p, P(vp), vp]
    L.tsdf_batch_create.argtypes = [ctypes.c_int32, P(vp)]
    L.tsdf_batch_destroy.argtypes = [vp]
    L.tsdf_batch_set_option.argtypes = [vp, ctypes.c_int32, ctypes.c_int64]
    L.tsdf_batch_get_config.argtypes = [vp] + [P(ctypes.c_int32)] * 8
    L.tsdf_batch_integrate.argtypes = [vp, P(vp), P(vp), P(i64), f32p, ctypes.c_int32, vp]
    L.tsdf_integrate_batch.argtypes = [P(vp), P(vp), P(i64), f32p, ctypes.c_int32, vp]
    L.tsdf_batch_sync.argtypes = [vp, vp]
    L.tsdf_server_create.argtypes = [P(tsdf_server_config), P(vp)]
    L.tsdf_server_destroy.argtypes = [vp]
    L.tsdf_server_open_session.argtypes = [vp, P(tsdf_params), P(ctypes.c_int32)]
    L.tsdf_server_close_session.argtypes = [vp, ctypes.c_int32]
    L.tsdf_server_submit.argtypes = [vp, ctypes.c_int32, vp, i64, f32p, P(i64), P(ctypes.c_uint64)]
    L.tsdf_server_submit_many.argtypes = [vp, ctypes.c_int32, P(ctypes.c_int32), P(vp), P(i64), f32p,
                                          P(ctypes.c_uint64), P(ctypes.c_int32)]
    L.tsdf_server_wait_many.argtypes = [vp, ctypes.c_int32, P(ctypes.c_uint64), P(tsdf_request_result), i64]
    L.tsdf_server_wait.argtypes = [vp, ctypes.c_uint64, P(tsdf_request_result), i64]
    L.tsdf_server_session_map.argtypes = [vp, ctypes.c_int32, P(vp)]
    L.tsdf_server_get_stats.argtypes = [vp, P(tsdf_server_stats)]
    L.tsdf_integrate_static.argtypes = [vp, P(tsdf_params), vp, i64, f32p, P(tsdf_scan_stats), vp]
    L.tsdf_error_string.argtypes = [i32]
    L.tsdf_error_string.restype = ctypes.c_char_p
    L.tsdf_last_cuda_error.argtypes = []
    for name in ("tsdf_map_create", "tsdf_map_destroy", "tsdf_integrate", "tsdf_integrate_host", "tsdf_shift",
                 "tsdf_read", "tsdf_write", "tsdf_stats", "tsdf_get_origin", "tsdf_grid_device_ptr",
                 "tsdf_last_cuda_error", "tsdf_profile_enable", "tsdf_profile_read", "tsdf_set_option",
                 "tsdf_integrate_static", "tsdf_probe_reduction_rate", "tsdf_map_save", "tsdf_map_load", "tsdf_extract_surface", "tsdf_map_device_bytes", "tsdf_register_system", "tsdf_register", "tsdf_extract_mesh", "tsdf_get_reduction", "tsdf_batch_create", "tsdf_batch_destroy", "tsdf_batch_set_option",
                 "tsdf_batch_get_config", "tsdf_batch_integrate", "tsdf_integrate_batch", "tsdf_batch_sync",
                 "tsdf_server_create", "tsdf_server_destroy", "tsdf_server_open_session", "tsdf_server_close_session",
                 "tsdf_server_submit", "tsdf_server_submit_many", "tsdf_server_wait", "tsdf_server_wait_many", "tsdf_server_session_map", "tsdf_server_get_stats"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def _check(rc: int, what: str):
    if rc != TSDF_OK:
        raise TsdfError(rc, what)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(p: dict) -> tsdf_params:
    s = tsdf_params()
    for a in range(3):
        s.dims[a] = int(p["dims"][a])
        s.origin[a] = int(p["origin"][a])
    s.voxel_size = float(p["voxel_size"])
    s.tau = float(p["tau"])
    s.w_max = int(p["w_max"])
    s.delta_z = float(p["delta_z"])
    s.r_min = float(p["r_min"])
    s.r_max = float(p["r_max"])
    s.reduce = int(p.get("reduce", 0))
    s.flags = int(p.get("flags", 0))
    return s


def _pose_arg(pose):
    a = np.ascontiguousarray(np.asarray(pose, dtype=np.float32).reshape(12))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _pose_addr(pose):
    """The pose as float32[12] (the array itself when it already is one, else a
    copy) and its address; the caller keeps the array alive over the call."""
    if not (isinstance(pose, np.ndarray) and pose.dtype == np.float32 and pose.size == 12
            and pose.flags.c_contiguous):
        pose = np.ascontiguousarray(np.asarray(pose, dtype=np.float32).reshape(12))
    return pose, pose.ctypes.data


def _i64_3(v):
    a = (ctypes.c_int64 * 3)(*[int(x) for x in v])
    return a


# ---- functions with the C ABI's names -------------------------------------

def tsdf_error_string(code: int) -> str:
    return lib().tsdf_error_string(int(code)).decode()


def tsdf_last_cuda_error() -> int:
    return int(lib().tsdf_last_cuda_error())


def tsdf_map_create(params: dict | tsdf_params) -> int:
    prm = params if isinstance(params, tsdf_params) else make_params(params)
    h = ctypes.c_void_p()
    _check(lib().tsdf_map_create(ctypes.byref(prm), ctypes.byref(h)), "tsdf_map_create")
    return h.value


def tsdf_map_destroy(handle: int) -> None:
    _check(lib().tsdf_map_destroy(handle), "tsdf_map_destroy")


def tsdf_integrate(handle: int, points_dev, n: int, pose, stream=None) -> None:
    """points_dev: a CUDA float32 tensor of shape (n, 4) (or a raw device pointer)."""
    ptr = points_dev if isinstance(points_dev, int) else points_dev.data_ptr()
    pa, pp = _pose_addr(pose)
    _check(lib().tsdf_integrate(handle, ptr, int(n), pp, _stream_ptr(stream)), "tsdf_integrate")


def tsdf_integrate_host(handle: int, points_host, n: int, pose, stream=None) -> None:
    """points_host: a host float32 array/tensor of shape (n, 4), pinned or pageable."""
    if isinstance(points_host, int):
        ptr = points_host
    elif isinstance(points_host, np.ndarray):
        assert points_host.dtype == np.float32 and points_host.flags.c_contiguous
        ptr = points_host.ctypes.data
    else:
        ptr = points_host.data_ptr()
    pa, pp = _pose_addr(pose)
    _check(lib().tsdf_integrate_host(handle, ptr, int(n), pp, _stream_ptr(stream)), "tsdf_integrate_host")


def tsdf_shift(handle: int, new_origin, stream=None) -> None:
    _check(lib().tsdf_shift(handle, _i64_3(new_origin), _stream_ptr(stream)), "tsdf_shift")


def tsdf_read(handle: int, lo, hi, stream=None):
    """Returns (value, weight) int16 numpy arrays of shape (z, y, x) for the global box [lo, hi)."""
    shape = (int(hi[2] - lo[2]), int(hi[1] - lo[1]), int(hi[0] - lo[0]))
    v = np.zeros(shape, dtype=np.int16)
    w = np.zeros(shape, dtype=np.int16)
    _check(lib().tsdf_read(handle, _i64_3(lo), _i64_3(hi), v.ctypes.data, w.ctypes.data, _stream_ptr(stream)),
           "tsdf_read")
    return v, w


def tsdf_write(handle: int, lo, hi, value, weight, stream=None) -> None:
    v = np.ascontiguousarray(value, dtype=np.int16)
    w = np.ascontiguousarray(weight, dtype=np.int16)
    _check(lib().tsdf_write(handle, _i64_3(lo), _i64_3(hi), v.ctypes.data, w.ctypes.data, _stream_ptr(stream)),
           "tsdf_write")


def tsdf_stats(handle: int, stream=None) -> dict:
    st = tsdf_scan_stats()
    _check(lib().tsdf_stats(handle, ctypes.byref(st), _stream_ptr(stream)), "tsdf_stats")
    return dict(valid_rays=st.valid_rays, hits=st.hits, touched=st.touched)


def tsdf_get_origin(handle: int):
    o = (ctypes.c_int64 * 3)()
    _check(lib().tsdf_get_origin(handle, o), "tsdf_get_origin")
    return tuple(int(x) for x in o)


def tsdf_grid_device_ptr(handle: int) -> int:
    p = ctypes.c_void_p()
    _check(lib().tsdf_grid_device_ptr(handle, ctypes.byref(p)), "tsdf_grid_device_ptr")
    return p.value


def tsdf_integrate_static(grid_dev, params, points_dev, n: int, pose, stream=None, want_stats: bool = True):
    """Integrate one scan into a caller-owned grid without any device allocation.

    grid_dev: CUDA int32/uint32 tensor (or device pointer) of dims product words;
    points_dev: CUDA float32 (n, 4) tensor (or device pointer). Returns the
    scan's counters (and synchronises the stream) when want_stats, else None.
    """
    prm = params if isinstance(params, tsdf_params) else make_params(params)
    # The caller owns the grid here, so nothing on the C side knows its size:
    # tensors are checked before their addresses are passed on (a raw pointer
    # is the caller's responsibility).
    if not isinstance(grid_dev, int):
        voxels = int(prm.dims[0]) * int(prm.dims[1]) * int(prm.dims[2])
        if (not grid_dev.is_cuda or not grid_dev.is_contiguous() or grid_dev.element_size() != 4
                or grid_dev.is_floating_point() or grid_dev.numel() != voxels):
            raise TsdfError(TSDF_ERR_INVALID, "tsdf_integrate_static: grid must be a contiguous 32-bit integer CUDA "
                                              f"tensor of {voxels} words")
    if not isinstance(points_dev, int):
        import torch
        if (not points_dev.is_cuda or not points_dev.is_contiguous() or points_dev.dtype != torch.float32
                or points_dev.dim() != 2 or points_dev.shape[1] != 4 or int(n) > points_dev.shape[0]):
            raise TsdfError(TSDF_ERR_INVALID, "tsdf_integrate_static: points must be a contiguous float32 (>= n, 4) "
                                              "CUDA tensor")
        if not isinstance(grid_dev, int) and points_dev.device != grid_dev.device:
            raise TsdfError(TSDF_ERR_INVALID, "tsdf_integrate_static: grid and points on different devices")
    for t in (grid_dev, points_dev):
        if not isinstance(t, int):
            import torch
            if t.device.index != torch.cuda.current_device():
                raise TsdfError(TSDF_ERR_INVALID, "tsdf_integrate_static: tensors must be on the current device")
    gptr = grid_dev if isinstance(grid_dev, int) else grid_dev.data_ptr()
    pptr = points_dev if isinstance(points_dev, int) else points_dev.data_ptr()
    pa, pp = _pose_arg(pose)
    st = tsdf_scan_stats()
    _check(lib().tsdf_integrate_static(gptr, ctypes.byref(prm), pptr, int(n), pp,
                                       ctypes.byref(st) if want_stats else None, _stream_ptr(stream)),
           "tsdf_integrate_static")
    return dict(valid_rays=st.valid_rays, hits=st.hits, touched=st.touched) if want_stats else None


def _batch_args(maps, points, poses):
    count = len(maps)
    assert len(points) == count and len(poses) == count
    mh = (ctypes.c_void_p * count)(*[m if isinstance(m, int) else m.handle for m in maps])
    ph = (ctypes.c_void_p * count)(*[p if isinstance(p, int) else p.data_ptr() for p in points])
    nn = (ctypes.c_int64 * count)(*[0 if isinstance(p, int) else int(p.shape[0]) for p in points])
    pa = np.ascontiguousarray(np.stack([np.asarray(x, np.float32).reshape(12) for x in poses]) if count else
                              np.zeros((0, 12), np.float32))
    return count, mh, ph, nn, pa


def tsdf_batch_create(max_count: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().tsdf_batch_create(int(max_count), ctypes.byref(h)), "tsdf_batch_create")
    return h.value


def tsdf_batch_destroy(batch: int) -> None:
    _check(lib().tsdf_batch_destroy(batch), "tsdf_batch_destroy")


def tsdf_batch_set_option(batch: int, option: int, value: int) -> None:
    _check(lib().tsdf_batch_set_option(batch, int(option), int(value)), "tsdf_batch_set_option")


def tsdf_batch_get_config(batch: int) -> dict:
    c, m, k, r, t, th, ct, ap = (ctypes.c_int32() for _ in range(8))
    _check(lib().tsdf_batch_get_config(batch, ctypes.byref(c), ctypes.byref(m), ctypes.byref(k), ctypes.byref(r),
                                       ctypes.byref(t), ctypes.byref(th), ctypes.byref(ct), ctypes.byref(ap)),
           "tsdf_batch_get_config")
    return dict(config=c.value, merge=m.value, steps_per_item=k.value, reduction=r.value, tuned=bool(t.value),
                threads_per_cta=th.value, ctas=ct.value, apply_voxel_pairs=ap.value)


def tsdf_batch_integrate(batch: int, maps, points, poses, stream=None) -> None:
    """maps: TsdfMap objects or handles; points: CUDA float32 (n_i, 4) tensors; poses: 12 floats each."""
    count, mh, ph, nn, pa = _batch_args(maps, points, poses)
    _check(lib().tsdf_batch_integrate(batch, mh, ph, nn, pa.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), count,
                                      _stream_ptr(stream)), "tsdf_batch_integrate")


def tsdf_integrate_batch(maps, points, poses, stream=None) -> None:
    count, mh, ph, nn, pa = _batch_args(maps, points, poses)
    _check(lib().tsdf_integrate_batch(mh, ph, nn, pa.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), count,
                                      _stream_ptr(stream)), "tsdf_integrate_batch")


def tsdf_batch_sync(batch: int, stream=None) -> int:
    """Waits; returns TSDF_OK or TSDF_ERR_TIMEOUT (a device barrier gave up). Other errors raise."""
    rc = lib().tsdf_batch_sync(batch, _stream_ptr(stream))
    if rc not in (TSDF_OK, TSDF_ERR_TIMEOUT):
        _check(rc, "tsdf_batch_sync")
    return rc


def tsdf_server_create(hbm_budget_bytes: int, max_points: int = 1 << 18, max_batch: int = 32, streams: int = 2,
                       max_outstanding: int = 64, store_chunks: int = 0) -> int:
    cfg = tsdf_server_config(int(hbm_budget_bytes), int(max_points), int(max_batch), int(streams),
                             int(max_outstanding), int(store_chunks))
    h = ctypes.c_void_p()
    _check(lib().tsdf_server_create(ctypes.byref(cfg), ctypes.byref(h)), "tsdf_server_create")
    return h.value


def tsdf_server_destroy(server: int) -> None:
    _check(lib().tsdf_server_destroy(server), "tsdf_server_destroy")


def tsdf_server_open_session(server: int, params) -> int:
    prm = params if isinstance(params, tsdf_params) else make_params(params)
    sid = ctypes.c_int32()
    _check(lib().tsdf_server_open_session(server, ctypes.byref(prm), ctypes.byref(sid)), "tsdf_server_open_session")
    return sid.value


def tsdf_server_close_session(server: int, session: int) -> None:
    _check(lib().tsdf_server_close_session(server, int(session)), "tsdf_server_close_session")


def tsdf_server_submit(server: int, session: int, points_host, pose, new_origin=None) -> int:
    """points_host: float32 (n, 4) host numpy array (copied before returning) or
    pinned CPU tensor (read in place: keep it unchanged until the ticket is
    waited for). Returns a ticket."""
    if isinstance(points_host, np.ndarray):
        pts = np.ascontiguousarray(points_host, dtype=np.float32).reshape(-1, 4)
        ptr, n = pts.ctypes.data, pts.shape[0]
    else:
        ptr, n = points_host.data_ptr(), points_host.shape[0]
    pa, pp = _pose_arg(pose)
    org = _i64_3(new_origin) if new_origin is not None else None
    t = ctypes.c_uint64()
    _check(lib().tsdf_server_submit(server, int(session), ptr, n, pp, org, ctypes.byref(t)), "tsdf_server_submit")
    return t.value


def tsdf_server_submit_many(server: int, sessions, points_host, poses):
    """Submit several scans in one call (pinned tensors read in place, numpy
    arrays copied). Returns the tickets of the scans queued: all of them, or a
    prefix when the server pushed back (TSDF_ERR_BUSY); other errors raise."""
    k = len(sessions)
    keep = []
    ptrs = (ctypes.c_void_p * k)()
    ns = (ctypes.c_int64 * k)()
    for i, p in enumerate(points_host):
        if isinstance(p, np.ndarray):
            p = np.ascontiguousarray(p, dtype=np.float32).reshape(-1, 4)
            keep.append(p)
            ptrs[i], ns[i] = p.ctypes.data, p.shape[0]
        else:
            ptrs[i], ns[i] = p.data_ptr(), p.shape[0]
    ses = (ctypes.c_int32 * k)(*[int(x) for x in sessions])
    pz = np.ascontiguousarray(np.asarray(poses, np.float32).reshape(k, 12))
    tk = (ctypes.c_uint64 * k)()
    done = ctypes.c_int32()
    rc = lib().tsdf_server_submit_many(server, k, ses, ptrs, ns, pz.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       tk, ctypes.byref(done))
    if rc not in (TSDF_OK, TSDF_ERR_BUSY):
        raise TsdfError(rc, "tsdf_server_submit_many")
    return list(tk)[:done.value]


def _result_dict(r) -> dict:
    return dict(ticket=r.ticket, session=r.session, status=r.status, batch_size=r.batch_size,
                stats=dict(valid_rays=r.stats.valid_rays, hits=r.stats.hits, touched=r.stats.touched),
                t_submit_us=r.t_submit_us, t_start_us=r.t_start_us, t_done_us=r.t_done_us)


def tsdf_server_wait(server: int, ticket: int, timeout_us: int = -1) -> dict:
    r = tsdf_request_result()
    rc = lib().tsdf_server_wait(server, ctypes.c_uint64(ticket), ctypes.byref(r), int(timeout_us))
    if rc != TSDF_OK:
        raise TsdfError(rc, "tsdf_server_wait")
    return _result_dict(r)


def tsdf_server_wait_many(server: int, tickets, timeout_us: int = -1) -> list:
    """Wait for several tickets in order (one call); returns one result dict per
    ticket. A dict's "status" is the request's status, or TSDF_ERR_TIMEOUT /
    TSDF_ERR_INVALID for a ticket that was not taken (a timed-out one stays
    pending)."""
    k = len(tickets)
    tk = (ctypes.c_uint64 * k)(*[int(t) for t in tickets])
    res = (tsdf_request_result * k)()
    lib().tsdf_server_wait_many(server, k, tk, res, int(timeout_us))
    return [_result_dict(r) for r in res]


def tsdf_server_session_map(server: int, session: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().tsdf_server_session_map(server, int(session), ctypes.byref(h)), "tsdf_server_session_map")
    return h.value


def tsdf_server_get_stats(server: int) -> dict:
    st = tsdf_server_stats()
    _check(lib().tsdf_server_get_stats(server, ctypes.byref(st)), "tsdf_server_get_stats")
    return dict(sessions=st.sessions, used_bytes=st.used_bytes, completed=st.completed, batches=st.batches,
                queued=st.queued, mean_batch=st.mean_batch)


def tsdf_set_option(handle: int, option: int, value: int) -> None:
    _check(lib().tsdf_set_option(handle, int(option), int(value)), "tsdf_set_option")


def tsdf_profile_enable(handle: int, enable: bool = True) -> None:
    _check(lib().tsdf_profile_enable(handle, 1 if enable else 0), "tsdf_profile_enable")


def tsdf_profile_read(handle: int) -> dict:
    """{kernel name: (launches, total_ms)} accumulated since profiling was enabled."""
    buf = (tsdf_kernel_time * 8)()
    cnt = ctypes.c_int32()
    _check(lib().tsdf_profile_read(handle, buf, 8, ctypes.byref(cnt)), "tsdf_profile_read")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(cnt.value)}


def tsdf_extract_surface(handle: int, min_weight: int = 1, out=None, stream=None):
    """Zero-crossing points of the window. out: CUDA float32 (cap, 4) tensor or
    None (sized automatically with a second call). Returns (points view, count)."""
    import torch
    cnt = ctypes.c_int64()
    if out is None:
        _check(lib().tsdf_extract_surface(handle, min_weight, None, 0, ctypes.byref(cnt), _stream_ptr(stream)),
               "tsdf_extract_surface")
        out = torch.empty((max(int(cnt.value), 1), 4), dtype=torch.float32, device="cuda")
    assert out.dtype == torch.float32 and out.is_contiguous() and out.shape[1] == 4
    _check(lib().tsdf_extract_surface(handle, min_weight, out.data_ptr(), out.shape[0], ctypes.byref(cnt),
                                      _stream_ptr(stream)), "tsdf_extract_surface")
    n = int(cnt.value)
    return out[:min(n, out.shape[0])], n


def tsdf_get_reduction(handle: int) -> int:
    out = ctypes.c_int32()
    _check(lib().tsdf_get_reduction(handle, ctypes.byref(out)), "tsdf_get_reduction")
    return int(out.value)


def tsdf_extract_mesh(handle: int, min_weight: int = 1, out=None, stream=None):
    """Marching-tetrahedra triangles of the window. out: CUDA float32 (cap, 3, 3)
    tensor or None (sized with a counting call first). Returns (triangles view, count)."""
    import torch
    cnt = ctypes.c_int64()
    if out is None:
        _check(lib().tsdf_extract_mesh(handle, min_weight, None, 0, ctypes.byref(cnt), _stream_ptr(stream)),
               "tsdf_extract_mesh")
        out = torch.empty((max(int(cnt.value), 1), 3, 3), dtype=torch.float32, device="cuda")
    assert out.dtype == torch.float32 and out.is_contiguous() and tuple(out.shape[1:]) == (3, 3)
    _check(lib().tsdf_extract_mesh(handle, min_weight, out.data_ptr(), out.shape[0], ctypes.byref(cnt),
                                   _stream_ptr(stream)), "tsdf_extract_mesh")
    n = int(cnt.value)
    return out[:min(n, out.shape[0])], n


def tsdf_register_system(handle: int, points_dev, pose, min_weight: int = 1, stream=None) -> np.ndarray:
    """Normal equations of scan-to-map registration at `pose`: float64[29]."""
    out = np.zeros(29, np.float64)
    pa, pp = _pose_arg(pose)
    _check(lib().tsdf_register_system(handle, points_dev.data_ptr(), points_dev.shape[0], pp, min_weight,
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_ptr(stream)),
           "tsdf_register_system")
    return out


def tsdf_register(handle: int, points_dev, pose, iterations: int = 10, min_weight: int = 1, stream=None):
    """Gauss-Newton scan-to-map registration from `pose`; returns (float32 pose[12], result dict)."""
    pose_a = (ctypes.c_float * 12)(*[float(x) for x in np.asarray(pose, np.float32).reshape(12)])
    res = tsdf_register_result()
    _check(lib().tsdf_register(handle, points_dev.data_ptr(), points_dev.shape[0], pose_a, iterations, min_weight,
                               ctypes.byref(res), _stream_ptr(stream)), "tsdf_register")
    return np.array(pose_a[:], np.float32), dict(used_points=res.used_points, rms=res.rms, step=res.step,
                                                  iterations=res.iterations)


def tsdf_map_device_bytes(handle: int) -> int:
    out = ctypes.c_int64()
    _check(lib().tsdf_map_device_bytes(handle, ctypes.byref(out)), "tsdf_map_device_bytes")
    return int(out.value)


class tsdf_store_stats(ctypes.Structure):
    _fields_ = [("device_chunks", ctypes.c_int64), ("device_capacity", ctypes.c_int64),
                ("host_chunks", ctypes.c_int64), ("host_capacity", ctypes.c_int64),
                ("spilled", ctypes.c_int64), ("dropped", ctypes.c_int64),
                ("file_chunks", ctypes.c_int64), ("to_file", ctypes.c_int64), ("from_file", ctypes.c_int64)]


def tsdf_map_reserve_store(handle: int, device_chunks: int) -> None:
    _check(lib().tsdf_map_reserve_store(handle, int(device_chunks)), "tsdf_map_reserve_store")


def tsdf_get_store_stats(handle: int) -> dict:
    st = tsdf_store_stats()
    _check(lib().tsdf_get_store_stats(handle, ctypes.byref(st)), "tsdf_get_store_stats")
    return {k: int(getattr(st, k)) for k, _ in tsdf_store_stats._fields_}


def tsdf_map_set_store_file(handle: int, path: str, host_chunks: int) -> None:
    _check(lib().tsdf_map_set_store_file(handle, os.fsencode(path), int(host_chunks)), "tsdf_map_set_store_file")


def tsdf_map_save(handle: int, path: str, stream=None) -> None:
    _check(lib().tsdf_map_save(handle, os.fsencode(path), _stream_ptr(stream)), "tsdf_map_save")


def tsdf_map_load(path: str, stream=None) -> int:
    h = ctypes.c_void_p()
    _check(lib().tsdf_map_load(os.fsencode(path), ctypes.byref(h), _stream_ptr(stream)), "tsdf_map_load")
    return h.value


FILE_HEADER_BYTES = 128
FILE_RECORD_BYTES = 2072


def _header_params(raw: np.ndarray) -> dict:
    if raw.size < FILE_HEADER_BYTES or bytes(raw[:8]) != b"TSDFMAP1":
        raise ValueError("not a map file")
    prm = tsdf_params.from_buffer_copy(raw[16:16 + ctypes.sizeof(tsdf_params)].tobytes())
    return dict(dims=tuple(prm.dims), voxel_size=prm.voxel_size, tau=prm.tau, w_max=prm.w_max,
                delta_z=prm.delta_z, r_min=prm.r_min, r_max=prm.r_max, reduce=prm.reduce, flags=prm.flags,
                origin=tuple(prm.origin))


def read_map_file(path: str):
    """Parse a map file (host only): (params dict, {chunk key: uint32[512] words})."""
    raw = np.fromfile(path, dtype=np.uint8)
    params = _header_params(raw)
    count = int(raw[88:96].view(np.int64)[0])
    recs = raw[FILE_HEADER_BYTES:].reshape(count, FILE_RECORD_BYTES)
    keys = recs[:, :24].copy().view(np.int64).reshape(count, 3)
    words = recs[:, 24:].copy().view(np.uint32).reshape(count, 512)
    return params, {tuple(int(x) for x in keys[i]): words[i] for i in range(count)}


def tsdf_probe_reduction_rate(pattern: int, stream=None) -> float:
    """Measured 64-bit L2 reduction rate (ops/s): pattern 0 coalesced, 1 scattered."""
    out = ctypes.c_double()
    _check(lib().tsdf_probe_reduction_rate(pattern, ctypes.byref(out), _stream_ptr(stream)), "tsdf_probe_reduction_rate")
    return out.value


# ---- convenience wrapper ---------------------------------------------------

class TsdfMap:
    """Owning wrapper of a tsdf_map handle."""

    def __init__(self, params: dict):
        self.params = dict(params)
        self.handle = tsdf_map_create(params)

    def close(self):
        if getattr(self, "handle", None):
            tsdf_map_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, points_dev, pose, stream=None):
        tsdf_integrate(self.handle, points_dev, points_dev.shape[0], pose, stream)

    def integrate_host(self, points_host, pose, stream=None):
        tsdf_integrate_host(self.handle, points_host, points_host.shape[0], pose, stream)

    def shift(self, new_origin, stream=None):
        tsdf_shift(self.handle, new_origin, stream)

    @property
    def origin(self):
        return tsdf_get_origin(self.handle)

    def read(self, lo=None, hi=None, stream=None):
        o = self.origin
        d = self.params["dims"]
        lo = o if lo is None else lo
        hi = tuple(o[a] + d[a] for a in range(3)) if hi is None else hi
        return tsdf_read(self.handle, lo, hi, stream)

    def write(self, value, weight, lo=None, hi=None, stream=None):
        o = self.origin
        d = self.params["dims"]
        lo = o if lo is None else lo
        hi = tuple(o[a] + d[a] for a in range(3)) if hi is None else hi
        tsdf_write(self.handle, lo, hi, value, weight, stream)

    def stats(self, stream=None):
        return tsdf_stats(self.handle, stream)

    def surface(self, min_weight: int = 1, stream=None):
        """Zero-crossing points (x, y, z, axis) as a CUDA float32 tensor."""
        return tsdf_extract_surface(self.handle, min_weight, None, stream)[0]

    def mesh(self, min_weight: int = 1, stream=None):
        """Marching-tetrahedra triangles (n, 3, 3) as a CUDA float32 tensor."""
        return tsdf_extract_mesh(self.handle, min_weight, None, stream)[0]

    def save(self, path: str, stream=None):
        tsdf_map_save(self.handle, path, stream)

    def set_store_file(self, path: str, host_chunks: int):
        """A file tier for the global store behind `host_chunks` host-memory chunks
        (`path` must not exist; it is removed when the map is closed)."""
        tsdf_map_set_store_file(self.handle, path, host_chunks)

    def store_stats(self) -> dict:
        return tsdf_get_store_stats(self.handle)

    @classmethod
    def load(cls, path: str, stream=None) -> "TsdfMap":
        """A new map from a file written by save()."""
        m = cls.__new__(cls)
        m.handle = tsdf_map_load(path, stream)
        m.params = _header_params(np.fromfile(path, dtype=np.uint8, count=FILE_HEADER_BYTES))
        return m
