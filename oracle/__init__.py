"""TEST INFRASTRUCTURE: Python binding of the CPU oracle (tsdf_oracle.cpp).

The oracle is a plain single-threaded C++ restatement of the paper's TSDF
integration (Section "TSDF Map Generation", Eq. 1 - Eq. 4) and of the local
map shift. It is used only by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline leg. It shares no code with the CUDA library and must
never be imported by the product path.

The shared library is compiled with g++ -ffp-contract=off so that no fused
multiply-add changes a float result; `build()` rebuilds it when the source is
newer than the binary.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsdf_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CXXFLAGS = ["-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-ffp-contract=off", "-fno-fast-math",
            "-fno-finite-math-only", "-fsigned-char"]


def build(force: bool = False) -> str:
    """Compile liboracle.so if missing or stale. Returns its path."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["g++", *CXXFLAGS, "-o", tmp, _SRC]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("voxel_size", ctypes.c_float), ("tau", ctypes.c_float),
                ("w_max", ctypes.c_int32), ("delta_z", ctypes.c_float), ("r_min", ctypes.c_float),
                ("r_max", ctypes.c_float), ("reduce", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("origin", ctypes.c_int64 * 3)]


def make_params(p: dict) -> OrcParams:
    o = OrcParams()
    for a in range(3):
        o.dims[a] = int(p["dims"][a])
        o.origin[a] = int(p["origin"][a])
    o.voxel_size = p["voxel_size"]
    o.tau = p["tau"]
    o.w_max = int(p["w_max"])
    o.delta_z = p["delta_z"]
    o.r_min = p["r_min"]
    o.r_max = p["r_max"]
    o.reduce = int(p.get("reduce", 0))
    o.flags = int(p.get("flags", 0))
    return o


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        vp, i64, f32p = ctypes.c_void_p, ctypes.c_int64, P(ctypes.c_float)
        L.orc_create.restype = vp
        L.orc_create.argtypes = [P(OrcParams)]
        L.orc_destroy.argtypes = [vp]
        L.orc_derived.argtypes = [P(OrcParams), f32p, f32p, P(ctypes.c_int32)]
        for name in ("orc_integrate", "orc_integrate_bruteforce"):
            fn = getattr(L, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [vp, f32p, i64, f32p]
        L.orc_integrate_parallel.restype = ctypes.c_int
        L.orc_integrate_parallel.argtypes = [vp, f32p, i64, f32p, ctypes.c_int32]
        L.orc_hits.restype = i64
        L.orc_hits.argtypes = [P(OrcParams), f32p, i64, f32p, P(i64), P(ctypes.c_int32), P(i64),
                               P(ctypes.c_int32), i64]
        L.orc_ray.argtypes = [f32p, f32p, ctypes.c_float, ctypes.c_float, ctypes.c_float, f32p]
        L.orc_quantize.restype = ctypes.c_int32
        L.orc_quantize.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float]
        for name in ("orc_eq12", "orc_eq12_scan"):
            getattr(L, name).argtypes = [ctypes.c_int32, ctypes.c_int32, i64, i64, ctypes.c_int32,
                                         P(ctypes.c_int32), P(ctypes.c_int32)]
        L.orc_shift.restype = ctypes.c_int
        L.orc_shift.argtypes = [vp, P(i64)]
        L.orc_read.restype = ctypes.c_int
        L.orc_read.argtypes = [vp, P(i64), P(i64), P(ctypes.c_int16), P(ctypes.c_int16)]
        L.orc_load_window.restype = ctypes.c_int
        L.orc_load_window.argtypes = [vp, P(ctypes.c_int16), P(ctypes.c_int16)]
        L.orc_origin.argtypes = [vp, P(i64)]
        L.orc_stats.argtypes = [vp, P(i64)]
        L.orc_store_chunks.restype = i64
        L.orc_store_chunks.argtypes = [vp]
        L.orc_register_system.restype = None
        L.orc_register_system.argtypes = [vp, f32p, i64, f32p, ctypes.c_int32, P(ctypes.c_double)]
        L.orc_mesh.restype = i64
        L.orc_mesh.argtypes = [vp, ctypes.c_int32, f32p, i64]
        L.orc_surface.restype = i64
        L.orc_surface.argtypes = [vp, ctypes.c_int32, f32p, i64]
        L.orc_global_chunks.restype = i64
        L.orc_global_chunks.argtypes = [vp, P(i64), P(ctypes.c_int16), P(ctypes.c_int16), i64]
        _lib = L
    return _lib


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def derived(p: dict):
    """(1/voxel_size, QMAX/tau, K) as the oracle derives them."""
    inv, qs, K = ctypes.c_float(), ctypes.c_float(), ctypes.c_int32()
    lib().orc_derived(ctypes.byref(make_params(p)), ctypes.byref(inv), ctypes.byref(qs), ctypes.byref(K))
    return inv.value, qs.value, K.value


def quantize(d: float, tau: float, qs: float) -> int:
    return int(lib().orc_quantize(d, tau, qs))


def eq12(gv, gw, S, W, w_max, scan_weight=False):
    """Eq. 1 / Eq. 2; scan_weight: the scan's average S/W as one observation."""
    nv, nw = ctypes.c_int32(), ctypes.c_int32()
    fn = lib().orc_eq12_scan if scan_weight else lib().orc_eq12
    fn(gv, gw, S, W, w_max, ctypes.byref(nv), ctypes.byref(nw))
    return nv.value, nw.value


def ray(pose, pt, r_min, r_max, delta_z):
    """Ray set-up of one point: dict(valid, fill, r, dir, ih)."""
    pose_a, pose_p = _f32(pose)
    pt_a, pt_p = _f32(np.asarray(pt, dtype=np.float32).reshape(4))
    out = np.zeros(9, dtype=np.float32)
    lib().orc_ray(pose_p, pt_p, r_min, r_max, delta_z, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return dict(valid=bool(out[0]), fill=bool(out[1]), r=out[2], dir=out[3:6].copy(), ih=out[6:9].copy())


def hits(p: dict, points: np.ndarray, pose: np.ndarray, cap: int | None = None, with_k: bool = False):
    """All contributions of a scan in enumeration order, in or out of the window.

    Returns (g int64[H,3], q int32[H], ray int64[H]) and, with_k, also the
    march step k int32[H] of each contribution."""
    pts_a, pts_p = _f32(points.reshape(-1, 4))
    pose_a, pose_p = _f32(pose)
    n = pts_a.shape[0]
    prm = make_params(p)
    P = ctypes.POINTER
    if cap is None:
        cap = int(lib().orc_hits(ctypes.byref(prm), pts_p, n, pose_p, None, None, None, None, 0))
    g = np.zeros((max(cap, 1), 3), dtype=np.int64)
    q = np.zeros(max(cap, 1), dtype=np.int32)
    r = np.zeros(max(cap, 1), dtype=np.int64)
    k = np.zeros(max(cap, 1), dtype=np.int32)
    cnt = lib().orc_hits(ctypes.byref(prm), pts_p, n, pose_p, g.ctypes.data_as(P(ctypes.c_int64)),
                         q.ctypes.data_as(P(ctypes.c_int32)), r.ctypes.data_as(P(ctypes.c_int64)),
                         k.ctypes.data_as(P(ctypes.c_int32)), cap)
    m = min(cnt, cap)
    if with_k:
        return g[:m], q[:m], r[:m], k[:m]
    return g[:m], q[:m], r[:m]


def pose_update(pose: np.ndarray, system: np.ndarray) -> tuple:
    """One Gauss-Newton step of scan-to-map registration: solve H xi = -g
    (Cholesky, float64) for xi = (w, v) and apply q' = Exp(w) q + v to the
    pose: R' = Exp(w) R, t' = Exp(w) t + v (Rodrigues). Returns (float32 pose
    12, xi)."""
    H = np.zeros((6, 6))
    k = 0
    for r in range(6):
        for c in range(r, 6):
            H[r, c] = H[c, r] = system[k]
            k += 1
    g = system[21:27]
    L = np.linalg.cholesky(H)
    xi = -np.linalg.solve(L.T, np.linalg.solve(L, g))
    w, v = xi[:3], xi[3:]
    th = float(np.linalg.norm(w))
    K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    if th < 1e-12:
        E = np.eye(3) + K
    else:
        E = np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * (K @ K)
    P = np.asarray(pose, np.float64).reshape(3, 4)
    R = E @ P[:, :3]
    t = E @ P[:, 3] + v
    return np.concatenate([R, t[:, None]], axis=1).astype(np.float32).reshape(12), xi


class OracleMap:
    """A TSDF window held on the host by the oracle."""

    def __init__(self, params: dict):
        self.params = dict(params)
        self._p = make_params(params)
        self.h = lib().orc_create(ctypes.byref(self._p))
        if not self.h:
            raise ValueError("oracle rejected the map parameters")

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def integrate(self, points: np.ndarray, pose: np.ndarray, bruteforce: bool = False, threads: int = 0):
        """One scan. threads > 0: the rays split over that many host threads
        (identical result); bruteforce: the voxel-major enumeration."""
        pts_a, pts_p = _f32(points.reshape(-1, 4))
        pose_a, pose_p = _f32(pose)
        if threads > 0:
            rc = lib().orc_integrate_parallel(self.h, pts_p, pts_a.shape[0], pose_p, threads)
            if rc != 0:
                raise ValueError("oracle integrate failed")
            return
        fn = lib().orc_integrate_bruteforce if bruteforce else lib().orc_integrate
        rc = fn(self.h, pts_p, pts_a.shape[0], pose_p)
        if rc != 0:
            raise ValueError("oracle integrate failed")

    def shift(self, new_origin):
        a, p = _i64(new_origin)
        if lib().orc_shift(self.h, p) != 0:
            raise ValueError("oracle shift rejected the origin")

    @property
    def origin(self):
        out = np.zeros(3, dtype=np.int64)
        lib().orc_origin(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        return tuple(int(x) for x in out)

    def read(self, lo=None, hi=None):
        """(value, weight) int16 arrays of shape (z, y, x) for the global box [lo, hi)."""
        o = self.origin
        d = self.params["dims"]
        lo = o if lo is None else lo
        hi = tuple(o[a] + d[a] for a in range(3)) if hi is None else hi
        shape = (hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0])
        v = np.zeros(shape, dtype=np.int16)
        w = np.zeros(shape, dtype=np.int16)
        la, lp = _i64(lo)
        ha, hp = _i64(hi)
        P = ctypes.POINTER
        rc = lib().orc_read(self.h, lp, hp, v.ctypes.data_as(P(ctypes.c_int16)), w.ctypes.data_as(P(ctypes.c_int16)))
        if rc != 0:
            raise ValueError("oracle read: box outside the window")
        return v, w

    def load_window(self, v: np.ndarray, w: np.ndarray):
        v = np.ascontiguousarray(v, dtype=np.int16)
        w = np.ascontiguousarray(w, dtype=np.int16)
        P = ctypes.POINTER
        lib().orc_load_window(self.h, v.ctypes.data_as(P(ctypes.c_int16)), w.ctypes.data_as(P(ctypes.c_int16)))

    def stats(self):
        out = np.zeros(3, dtype=np.int64)
        lib().orc_stats(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        return dict(valid_rays=int(out[0]), hits=int(out[1]), touched=int(out[2]))

    def store_chunks(self) -> int:
        return int(lib().orc_store_chunks(self.h))

    def surface(self, min_weight: int = 1) -> np.ndarray:
        """Zero-crossing points of the window: float32 (n, 4) = (x, y, z, axis), z-y-x-axis order."""
        n = int(lib().orc_surface(self.h, min_weight, None, 0))
        out = np.zeros((max(n, 1), 4), np.float32)
        lib().orc_surface(self.h, min_weight, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n)
        return out[:n]

    def register_system(self, points: np.ndarray, pose: np.ndarray, min_weight: int = 1) -> np.ndarray:
        """Normal equations of scan-to-map registration at `pose`: float64[29] =
        H (21 upper-triangle entries, row by row), g (6), cost, point count."""
        pts_a, pts_p = _f32(points.reshape(-1, 4))
        pose_a, pose_p = _f32(pose)
        out = np.zeros(29, np.float64)
        lib().orc_register_system(self.h, pts_p, pts_a.shape[0], pose_p, min_weight,
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def mesh(self, min_weight: int = 1) -> np.ndarray:
        """Marching-tetrahedra triangles of the window's zero level set: float32 (n, 3, 3)."""
        n = int(lib().orc_mesh(self.h, min_weight, None, 0))
        out = np.zeros((max(n, 1), 3, 3), np.float32)
        lib().orc_mesh(self.h, min_weight, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n)
        return out[:n]

    def global_chunks(self):
        """Non-empty 8^3 chunks of the global map (window + store):
        {chunk key (x, y, z): (value int16[512], weight int16[512])}, cells in
        (z * 8 + y) * 8 + x order."""
        P = ctypes.POINTER
        n = int(lib().orc_global_chunks(self.h, None, None, None, 0))
        keys = np.zeros((max(n, 1), 3), np.int64)
        v = np.zeros((max(n, 1), 512), np.int16)
        w = np.zeros((max(n, 1), 512), np.int16)
        lib().orc_global_chunks(self.h, keys.ctypes.data_as(P(ctypes.c_int64)), v.ctypes.data_as(P(ctypes.c_int16)),
                                w.ctypes.data_as(P(ctypes.c_int16)), n)
        return {tuple(int(x) for x in keys[i]): (v[i], w[i]) for i in range(n)}
