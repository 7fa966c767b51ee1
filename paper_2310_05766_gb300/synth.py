"""Seeded synthetic LiDAR workloads: scenes, ray casting, noise and trajectories.

This module produces INPUTS only (sensor-frame point clouds, poses and the
map parameters of each workload). It holds none of the TSDF method's
arithmetic: no transform, no ray march, no distance, no update. Both the CUDA
path and the CPU oracle consume exactly the arrays made here.

Everything is deterministic from an integer seed. Random numbers come from a
SplitMix64 counter generator (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) and Gaussian samples from the
Box-Muller transform, both written out below, so the streams do not depend on
numpy's own generator versions. Ray casting is done in float64 against
analytic primitives and the result is rounded once to float32.

The sensor model is a structured (ordered) spinning LiDAR: points are stored
beam-major, row = scan line, column = azimuth, the ordered layout the paper's
front end relies on (Section "Related Work", structured point clouds). A beam
without a return yields a NaN point, which the method skips.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream (64-bit state, golden-ratio increment)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.state + idx * _GAMMA
            self.state = self.state + np.uint64(n) * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi)."""
        return lo + np.floor(self.uniform(n) * (hi - lo)).astype(np.int64)


# --------------------------------------------------------------------------
# Sensor model
# --------------------------------------------------------------------------

def beam_directions(n_beams: int, n_az: int, elev_lo_deg: float, elev_hi_deg: float) -> np.ndarray:
    """Unit directions in the sensor frame, shape (n_beams * n_az, 3), beam-major.

    Elevations are uniform over [lo, hi] inclusive; azimuths step 2*pi/n_az.
    """
    if n_beams == 1:
        elev = np.array([math.radians(0.5 * (elev_lo_deg + elev_hi_deg))])
    else:
        elev = np.radians(np.linspace(elev_lo_deg, elev_hi_deg, n_beams))
    az = 2.0 * math.pi * np.arange(n_az) / n_az
    ce, se = np.cos(elev)[:, None], np.sin(elev)[:, None]
    d = np.empty((n_beams, n_az, 3))
    d[..., 0] = ce * np.cos(az)[None, :]
    d[..., 1] = ce * np.sin(az)[None, :]
    d[..., 2] = se
    return d.reshape(-1, 3)


def rot_zyx(yaw: float, pitch: float = 0.0, roll: float = 0.0) -> np.ndarray:
    """Rotation matrix R = Rz(yaw) @ Ry(pitch) @ Rx(roll), float64."""
    cy, sy = math.cos(yaw), math.sin(yaw)
    cp, sp = math.cos(pitch), math.sin(pitch)
    cr, sr = math.cos(roll), math.sin(roll)
    rz = np.array([[cy, -sy, 0], [sy, cy, 0], [0, 0, 1.0]])
    ry = np.array([[cp, 0, sp], [0, 1.0, 0], [-sp, 0, cp]])
    rx = np.array([[1.0, 0, 0], [0, cr, -sr], [0, sr, cr]])
    return rz @ ry @ rx


def pose12(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Row-major 3x4 sensor-to-world pose [R | t] as float32[12]."""
    m = np.zeros((3, 4), dtype=np.float64)
    m[:, :3] = R
    m[:, 3] = t
    return m.astype(np.float32).reshape(12)


# --------------------------------------------------------------------------
# Analytic scene primitives (float64 ray casting)
# --------------------------------------------------------------------------

def _safe_div(a, b):
    with np.errstate(divide="ignore", invalid="ignore"):
        return a / b


def _box_entry(o, d, lo, hi):
    """Entry distance of rays o + s d into a solid axis-aligned box (inf if none)."""
    inv = _safe_div(1.0, d)
    t1 = (lo[None, :] - o[None, :]) * inv
    t2 = (hi[None, :] - o[None, :]) * inv
    with np.errstate(invalid="ignore"):
        tmin = np.nanmax(np.minimum(t1, t2), axis=1)
        tmax = np.nanmin(np.maximum(t1, t2), axis=1)
    hit = (tmax >= tmin) & (tmin > 0.0)
    return np.where(hit, tmin, np.inf)


def _box_exit(o, d, lo, hi):
    """Exit distance of rays starting inside a hollow box (a room's walls)."""
    inv = _safe_div(1.0, d)
    t1 = (lo[None, :] - o[None, :]) * inv
    t2 = (hi[None, :] - o[None, :]) * inv
    with np.errstate(invalid="ignore"):
        tfar = np.where(d > 0, t2, np.where(d < 0, t1, np.inf))
    return np.min(tfar, axis=1)


def _cyl_entry(o, d, cx, cy, rad, z0, z1):
    """Entry distance into a solid vertical cylinder with a top cap."""
    ox, oy = o[0] - cx, o[1] - cy
    a = d[:, 0] ** 2 + d[:, 1] ** 2
    b = 2.0 * (ox * d[:, 0] + oy * d[:, 1])
    c = ox * ox + oy * oy - rad * rad
    disc = b * b - 4.0 * a * c
    out = np.full(d.shape[0], np.inf)
    ok = (disc >= 0) & (a > 1e-300)
    s = np.where(ok, (-b - np.sqrt(np.where(ok, disc, 0.0))) / np.where(ok, 2.0 * a, 1.0), np.inf)
    z = o[2] + s * d[:, 2]
    side = ok & (s > 0) & (z >= z0) & (z <= z1)
    out = np.where(side, s, out)
    # top cap, seen from above
    with np.errstate(divide="ignore", invalid="ignore"):
        st = (z1 - o[2]) / d[:, 2]
    px = ox + st * d[:, 0]
    py = oy + st * d[:, 1]
    cap = (o[2] > z1) & (d[:, 2] < 0) & (st > 0) & (px * px + py * py <= rad * rad)
    return np.where(cap & (st < out), st, out)


def _plane_z(o, d, zg):
    """Hit distance with the horizontal plane z = zg from above."""
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (zg - o[2]) / d[:, 2]
    return np.where((d[:, 2] < 0) & (s > 0), s, np.inf)


@dataclass
class Scene:
    """A set of analytic primitives. Boxes and cylinders are solid."""

    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 6)))     # lo(3), hi(3)
    cylinders: np.ndarray = field(default_factory=lambda: np.zeros((0, 5)))  # cx, cy, r, z0, z1
    ground_z: float | None = None
    room: np.ndarray | None = None  # hollow enclosing box lo(3), hi(3); rays exit through it

    def cast(self, o: np.ndarray, d: np.ndarray, r_max: float = np.inf) -> np.ndarray:
        """Distance along unit rays d from origin o to the first surface (inf if none)."""
        o = np.asarray(o, dtype=np.float64)
        n = d.shape[0]
        best = np.full(n, np.inf)
        if self.room is not None:
            best = np.minimum(best, _box_exit(o, d, self.room[:3], self.room[3:]))
        if self.ground_z is not None:
            best = np.minimum(best, _plane_z(o, d, self.ground_z))
        # azimuth culling: each object only against the rays within its angular extent
        az = np.arctan2(d[:, 1], d[:, 0])
        order = np.argsort(az, kind="stable")
        az_sorted = az[order]

        def candidates(cx, cy, radius):
            dx, dy = cx - o[0], cy - o[1]
            dist = math.hypot(dx, dy)
            if dist - radius > r_max:
                return None
            if dist <= radius * 1.0001 + 1e-9:
                return np.arange(n)
            half = math.asin(min(1.0, radius / dist)) + 1e-6
            c = math.atan2(dy, dx)
            lo, hi = c - half, c + half
            parts = []
            for a, b in ((lo, hi), (lo + 2 * math.pi, hi + 2 * math.pi), (lo - 2 * math.pi, hi - 2 * math.pi)):
                i0 = np.searchsorted(az_sorted, a, side="left")
                i1 = np.searchsorted(az_sorted, b, side="right")
                if i1 > i0:
                    parts.append(order[i0:i1])
            if not parts:
                return None
            return np.concatenate(parts)

        for bx in self.boxes:
            lo, hi = bx[:3], bx[3:]
            cx, cy = 0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1])
            rad = 0.5 * math.hypot(hi[0] - lo[0], hi[1] - lo[1])
            idx = candidates(cx, cy, rad)
            if idx is None:
                continue
            t = _box_entry(o, d[idx], lo, hi)
            best[idx] = np.minimum(best[idx], t)
        for cyl in self.cylinders:
            cx, cy, rad, z0, z1 = cyl
            idx = candidates(cx, cy, rad)
            if idx is None:
                continue
            t = _cyl_entry(o, d[idx], cx, cy, rad, z0, z1)
            best[idx] = np.minimum(best[idx], t)
        return best

    def sdf(self, q: np.ndarray) -> np.ndarray:
        """Unsigned distance (float64) from points q (M,3) to the nearest surface.

        Used only by accuracy checks. Solid boxes and the room use exact
        axis-aligned box distances; cylinders use the exact capped-cylinder
        distance; the ground is |z - ground_z|.
        """
        q = np.asarray(q, dtype=np.float64)
        best = np.full(q.shape[0], np.inf)
        if self.room is not None:
            lo, hi = self.room[:3], self.room[3:]
            inner = np.minimum(q - lo[None, :], hi[None, :] - q)  # distance to each wall pair
            best = np.minimum(best, np.abs(inner).min(axis=1))
        if self.ground_z is not None:
            best = np.minimum(best, np.abs(q[:, 2] - self.ground_z))
        for bx in self.boxes:
            lo, hi = bx[:3], bx[3:]
            c, h = 0.5 * (lo + hi), 0.5 * (hi - lo)
            p = np.abs(q - c[None, :]) - h[None, :]
            outside = np.linalg.norm(np.maximum(p, 0.0), axis=1)
            inside = np.minimum(p.max(axis=1), 0.0)
            best = np.minimum(best, np.abs(outside + inside))
        for cyl in self.cylinders:
            cx, cy, rad, z0, z1 = cyl
            rr = np.hypot(q[:, 0] - cx, q[:, 1] - cy) - rad
            zc, zh = 0.5 * (z0 + z1), 0.5 * (z1 - z0)
            dz = np.abs(q[:, 2] - zc) - zh
            outside = np.hypot(np.maximum(rr, 0), np.maximum(dz, 0))
            inside = np.minimum(np.maximum(rr, dz), 0.0)
            best = np.minimum(best, np.abs(outside + inside))
        return best


# --------------------------------------------------------------------------
# Scans
# --------------------------------------------------------------------------

def make_scan(scene: Scene, R: np.ndarray, t: np.ndarray, dirs_sensor: np.ndarray,
              sigma: float, rng: SplitMix64, r_max: float) -> np.ndarray:
    """Cast the sensor's beams from pose (R, t) and return float32 (M, 4) sensor-frame points.

    Range noise is Gaussian with std sigma, truncated at +-3 sigma. Beams with
    no return within r_max give NaN points. Column 3 is 0 (unused).
    """
    dw = dirs_sensor @ np.asarray(R, dtype=np.float64).T
    rng_true = scene.cast(np.asarray(t, dtype=np.float64), dw, r_max=r_max)
    noise = np.clip(rng.normal(dirs_sensor.shape[0]), -3.0, 3.0) * sigma
    miss = ~np.isfinite(rng_true) | (rng_true > r_max)
    rho = np.where(miss, 0.0, rng_true + noise)
    pts = np.zeros((dirs_sensor.shape[0], 4), dtype=np.float64)
    pts[:, :3] = dirs_sensor * rho[:, None]
    pts[miss, :3] = np.nan
    return pts.astype(np.float32)


# --------------------------------------------------------------------------
# Map parameters and window placement
# --------------------------------------------------------------------------

QMAX = 32767


def delta_z_for(vfov_deg: float, hlines: int) -> float:
    """Eq. 3 evaluated in float64 on the host: tan(deg2rad(vfov / hlines)), rounded to float32."""
    return float(np.float32(math.tan(math.radians(vfov_deg / hlines))))


def params_dict(dims, voxel_size, tau, w_max, delta_z, r_min, r_max, reduce=0, origin=(0, 0, 0), flags=0):
    return dict(dims=tuple(int(x) for x in dims), voxel_size=float(np.float32(voxel_size)),
                tau=float(np.float32(tau)), w_max=int(w_max), delta_z=float(np.float32(delta_z)),
                r_min=float(np.float32(r_min)), r_max=float(np.float32(r_max)), reduce=int(reduce),
                origin=tuple(int(x) for x in origin), flags=int(flags))


def window_origin(center_xyz, dims, voxel_size) -> tuple:
    """Origin (voxel coords, multiples of 8) of a window of `dims` centred on a world point."""
    out = []
    for c, n in zip(center_xyz, dims):
        g = math.floor(float(c) / float(voxel_size)) - n // 2
        out.append(int(math.floor(g / 8.0) * 8))
    return tuple(out)


@dataclass
class Workload:
    name: str
    params: dict
    scans: list            # list of float32 (M, 4)
    poses: list            # list of float32[12]
    origins: list          # window origin to use for each scan (shift before integrating when it changes)
    scene: Scene | None = None
    meta: dict = field(default_factory=dict)


def _n_az_dirs(beams, az, lo, hi):
    return beam_directions(beams, az, lo, hi)


# --------------------------------------------------------------------------
# Workload 1: box room, one scan (16 x 360 beams)
# --------------------------------------------------------------------------

def box_room_scene() -> Scene:
    return Scene(boxes=np.array([[2.0, -0.5, -1.5, 3.0, 0.5, -0.5]]),
                 room=np.array([-5.0, -5.0, -1.5, 5.0, 5.0, 1.5]))


def workload_room(seed: int = 1, reduce: int = 0) -> Workload:
    """16 beams over [-15, 15] deg x 360 azimuths in a 10 x 10 x 3 m room with a 1 m box.

    Grid 256 x 256 x 64 at 0.05 m centred on the sensor, tau 0.2 m, Wmax 64,
    delta_z = tan(30/16 deg), sigma 0.01 m, one scan from the origin.
    """
    scene = box_room_scene()
    dirs = beam_directions(16, 360, -15.0, 15.0)
    rng = SplitMix64(seed)
    R = np.eye(3)
    t = np.zeros(3)
    pts = make_scan(scene, R, t, dirs, 0.01, rng, r_max=20.0)
    dims = (256, 256, 64)
    origin = window_origin((0.0, 0.0, 0.0), dims, 0.05)
    p = params_dict(dims, 0.05, 0.2, 64, delta_z_for(30.0, 16), 0.3, 20.0, reduce, origin)
    return Workload("box_room_16x360", p, [pts], [pose12(R, t)], [origin], scene,
                    meta=dict(beams=16, azimuths=360, seed=seed))


# --------------------------------------------------------------------------
# Workload 2: outdoor OS1-128-shaped sequence
# --------------------------------------------------------------------------

def _smooth_heading(rng: SplitMix64, n: int, dt: float):
    amp = rng.uniform(3, 0.05, 0.35)
    freq = rng.uniform(3, 0.02, 0.2)
    phase = rng.uniform(3, 0.0, 2 * math.pi)
    psi0 = float(rng.uniform(1, -math.pi, math.pi)[0])
    ts = np.arange(n) * dt
    psi = psi0 + sum(a * np.sin(2 * math.pi * f * ts + ph) for a, f, ph in zip(amp, freq, phase))
    return psi


def trajectory(n: int, speed: float, dt: float, seed: int, wobble_deg: float = 0.5,
               lateral: float = 0.0, straight_x: bool = False):
    """Seeded smooth ground-vehicle trajectory. Returns lists of (R, t) in float64.

    Heading is a sum of three seeded sinusoids (or +x when straight_x), small
    seeded roll/pitch wobble, and an optional lateral sinusoidal wiggle.
    """
    rng = SplitMix64(seed * 7919 + 13)
    psi = np.zeros(n) if straight_x else _smooth_heading(rng, n, dt)
    wob_f = rng.uniform(2, 0.1, 0.5)
    wob_p = rng.uniform(2, 0.0, 2 * math.pi)
    lat_f = float(rng.uniform(1, 0.1, 0.3)[0])
    pos = np.zeros(3)
    out = []
    for i in range(n):
        ts = i * dt
        pitch = math.radians(wobble_deg) * math.sin(2 * math.pi * wob_f[0] * ts + wob_p[0])
        roll = math.radians(wobble_deg) * math.sin(2 * math.pi * wob_f[1] * ts + wob_p[1])
        R = rot_zyx(float(psi[i]), pitch, roll)
        t = pos.copy()
        if lateral:
            t[1] += lateral * math.sin(2 * math.pi * lat_f * ts)
        out.append((R, t))
        pos = pos + speed * dt * np.array([math.cos(psi[i]), math.sin(psi[i]), 0.0])
    return out


def outdoor_scene(seed: int, path_xy: np.ndarray, n_boxes: int = 200, n_cyl: int = 50,
                  extent: float = 100.0, band: float = 4.0, ground_z: float = -1.8) -> Scene:
    """Ground plane + seeded boxes (sides U[0.5, 8]) + cylinders (r U[0.2, 1], h U[2, 8]).

    Object footprints within `band` metres of the path are rejected and redrawn.
    """
    rng = SplitMix64(seed)

    def far_from_path(cx, cy, rad):
        dd = np.hypot(path_xy[:, 0] - cx, path_xy[:, 1] - cy)
        return dd.min() > band + rad

    boxes = []
    while len(boxes) < n_boxes:
        c = rng.uniform(2, -extent, extent)
        s = rng.uniform(3, 0.5, 8.0)
        if not far_from_path(c[0], c[1], 0.5 * math.hypot(s[0], s[1])):
            continue
        boxes.append([c[0] - s[0] / 2, c[1] - s[1] / 2, ground_z, c[0] + s[0] / 2, c[1] + s[1] / 2, ground_z + s[2]])
    cyls = []
    while len(cyls) < n_cyl:
        c = rng.uniform(2, -extent, extent)
        rad = float(rng.uniform(1, 0.2, 1.0)[0])
        h = float(rng.uniform(1, 2.0, 8.0)[0])
        if not far_from_path(c[0], c[1], rad):
            continue
        cyls.append([c[0], c[1], rad, ground_z, ground_z + h])
    return Scene(boxes=np.array(boxes), cylinders=np.array(cyls), ground_z=ground_z)


def _recentre_origins(poses, dims, vs, threshold):
    origins = []
    centre = None
    cur = None
    for _, t in poses:
        if centre is None or math.hypot(t[0] - centre[0], t[1] - centre[1]) >= threshold:
            centre = t.copy()
            cur = window_origin(t, dims, vs)
        origins.append(cur)
    return origins


def workload_outdoor(n_scans: int = 100, seed: int = 2, reduce: int = 0, beams: int = 128,
                     azimuths: int = 1024, dims=(512, 512, 128), voxel_size: float = 0.064,
                     tau: float = 0.6, scene_seed: int | None = None) -> Workload:
    """OS1-128-shaped sequence: 128 beams over [-22.5, 22.5] deg x 1024 azimuths,
    range [0.5, 100] m, sigma 0.01 m, 10 Hz at 1 m/s, window 512 x 512 x 128 at
    0.064 m re-centred (origin snapped to 8 voxels) after each 1 m of motion.
    """
    poses = trajectory(n_scans, 1.0, 0.1, seed)
    path = np.array([t[:2] for _, t in poses])
    scene = outdoor_scene(seed if scene_seed is None else scene_seed, path)
    dirs = beam_directions(beams, azimuths, -22.5, 22.5)
    rng = SplitMix64(seed * 1000003 + 1)
    scans = [make_scan(scene, R, t, dirs, 0.01, rng, r_max=100.0) for R, t in poses]
    origins = _recentre_origins(poses, dims, voxel_size, 1.0)
    p = params_dict(dims, voxel_size, tau, 64, delta_z_for(45.0, beams), 0.5, 100.0, reduce, origins[0])
    return Workload(f"outdoor_{beams}x{azimuths}_seq{n_scans}", p, scans,
                    [pose12(R, t) for R, t in poses], origins, scene,
                    meta=dict(beams=beams, azimuths=azimuths, seed=seed))


# --------------------------------------------------------------------------
# Workload 3: batch of independent maps of uneven sizes
# --------------------------------------------------------------------------

def workload_batch(n_maps: int = 64, seed: int = 3, reduce: int = 0, dims_choices=None):
    """One scan per map; beams in {16,32,64,128} x azimuths in {512,1024,2048},
    grids in {256^3, 512x512x128} at 0.064 m, tau 0.6 m, per-map scene seed."""
    rng = SplitMix64(seed)
    beams_c = [16, 32, 64, 128]
    az_c = [512, 1024, 2048]
    dims_c = dims_choices or [(256, 256, 256), (512, 512, 128)]
    out = []
    for i in range(n_maps):
        b = beams_c[int(rng.integers(1, 0, 4)[0])]
        a = az_c[int(rng.integers(1, 0, 3)[0])]
        dims = dims_c[int(rng.integers(1, 0, len(dims_c))[0])]
        w = workload_outdoor(n_scans=1, seed=1000 + seed * 100 + i, reduce=reduce, beams=b, azimuths=a,
                             dims=dims, voxel_size=0.064, tau=0.6)
        w.name = f"batch{i}_{b}x{a}_{dims[0]}x{dims[1]}x{dims[2]}"
        out.append(w)
    return out


# --------------------------------------------------------------------------
# Workload 4: high-resolution corridor
# --------------------------------------------------------------------------

def corridor_scene(seed: int, n_boxes: int = 200) -> Scene:
    """Corridor: walls y = +-1.5, floor z = -1.2, ceiling z = 1.8, x in [-100, 100],
    with seeded small boxes (sides U[0.1, 0.6]) standing against the walls."""
    rng = SplitMix64(seed)
    boxes = []
    for _ in range(n_boxes):
        x = float(rng.uniform(1, -99.0, 99.0)[0])
        s = rng.uniform(3, 0.1, 0.6)
        side = 1.0 if rng.uniform(1)[0] < 0.5 else -1.0
        if side > 0:
            y0, y1 = 1.5 - s[1], 1.5
        else:
            y0, y1 = -1.5, -1.5 + s[1]
        boxes.append([x - s[0] / 2, y0, -1.2, x + s[0] / 2, y1, -1.2 + s[2]])
    return Scene(boxes=np.array(boxes), room=np.array([-100.0, -1.5, -1.2, 100.0, 1.5, 1.8]))


def workload_corridor(n_scans: int = 50, seed: int = 4, reduce: int = 0, beams: int = 128,
                      azimuths: int = 2048, dims=(1024, 1024, 256)) -> Workload:
    """128 x 2048 beams over [-22.5, 22.5] deg, 0.02 m voxels, 1024 x 1024 x 256 grid,
    tau 0.1 m, 10 Hz at 0.5 m/s along +x with a +-0.2 m lateral wiggle, window
    re-centred after each 0.5 m."""
    scene = corridor_scene(seed)
    poses = trajectory(n_scans, 0.5, 0.1, seed, wobble_deg=0.3, lateral=0.2, straight_x=True)
    dirs = beam_directions(beams, azimuths, -22.5, 22.5)
    rng = SplitMix64(seed * 1000003 + 1)
    scans = [make_scan(scene, R, t, dirs, 0.01, rng, r_max=100.0) for R, t in poses]
    origins = _recentre_origins(poses, dims, 0.02, 0.5)
    p = params_dict(dims, 0.02, 0.1, 64, delta_z_for(45.0, beams), 0.5, 100.0, reduce, origins[0])
    return Workload(f"corridor_{beams}x{azimuths}_seq{n_scans}", p, scans,
                    [pose12(R, t) for R, t in poses], origins, scene,
                    meta=dict(beams=beams, azimuths=azimuths, seed=seed))


# --------------------------------------------------------------------------
# Workload 5: serving sessions
# --------------------------------------------------------------------------

def serving_sessions(n_sessions: int = 32, seed: int = 100):
    """Per-session map parameters: dims in {256^3, 512x512x128}, voxel in
    {0.05, 0.064, 0.08, 0.1} m, tau U[0.2, 0.6] m (at least 2 voxels)."""
    out = []
    for i in range(n_sessions):
        rng = SplitMix64(seed + i)
        dims = [(256, 256, 256), (512, 512, 128)][int(rng.integers(1, 0, 2)[0])]
        vs = [0.05, 0.064, 0.08, 0.1][int(rng.integers(1, 0, 4)[0])]
        tau = max(float(rng.uniform(1, 0.2, 0.6)[0]), 2 * vs)
        out.append(dict(dims=dims, voxel_size=vs, tau=tau, seed=seed + i))
    return out


def poisson_arrivals(rate_hz: float, duration_s: float, n_sessions: int, seed: int):
    """Arrival times (s) and session ids of a Poisson process with the given aggregate rate."""
    rng = SplitMix64(seed)
    times, sess = [], []
    tcur = 0.0
    while True:
        u = float(rng.uniform(1)[0])
        tcur += -math.log1p(-u) / rate_hz
        if tcur >= duration_s:
            break
        times.append(tcur)
        sess.append(int(rng.integers(1, 0, n_sessions)[0]))
    return np.array(times), np.array(sess, dtype=np.int64)
