"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
golden values (tests/golden/), closed forms for axis-aligned rays, an FP64
analytic signed distance field, a brute-force voxel-major enumeration in a
different loop order, textbook reductions (numpy min / sums) over the raw
contribution list, and invariants of Eq. 1 / Eq. 2 and of the map shift.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2310_05766_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            rows.append(line.split())
    return rows


# ---------------------------------------------------------------- constants

@pytest.mark.parametrize("vs,tau,K", [(0.05, 0.2, 4), (0.064, 0.6, 9), (0.02, 0.1, 5), (0.125, 0.5, 4),
                                      (0.1, 0.2, 2), (0.08, 0.6, 7)])
def test_march_step_count(vs, tau, K):
    """K = floor(tau / voxel): the march covers +-tau around the hit in voxel steps."""
    p = synth.params_dict((8, 8, 8), vs, tau, 64, 0.0, 0.1, 10.0)
    assert oracle.derived(p)[2] == K


# ---------------------------------------------------------------- Eq. 1 / Eq. 2

def test_eq12_golden_table():
    """Eq. 1 / Eq. 2 against the hand-computed table (tests/golden/eq12_table.txt)."""
    rows = _table("eq12_table.txt")
    assert len(rows) >= 15
    for r in rows:
        gv, gw, S, W, wmax, ev, ew = (int(x) for x in r)
        assert oracle.eq12(gv, gw, S, W, wmax) == (ev, ew), r


def test_eq12_exact_rational_rounding():
    """Random Eq. 1 cases against exact rational arithmetic, rounding half away from zero."""
    rng = np.random.default_rng(5)
    for _ in range(3000):
        gv = int(rng.integers(-32767, 32768))
        gw = int(rng.integers(0, 65))
        W = int(rng.integers(1, 200))
        S = int(rng.integers(-32767, 32768)) * W // max(1, int(rng.integers(1, 4)))
        S = max(-32767 * W, min(32767 * W, S))
        wmax = int(rng.integers(1, 65))
        x = Fraction(gv * gw + S, gw + W)
        mag = abs(x)
        expect = int(mag + Fraction(1, 2)) if mag.denominator != 1 else int(mag)
        expect = expect if x >= 0 else -expect
        nv, nw = oracle.eq12(gv, gw, S, W, wmax)
        assert nv == expect
        assert nw == min(wmax, gw + W)
        assert -32767 <= nv <= 32767


# ---------------------------------------------------------------- quantiser

def test_quantize_ties_golden():
    tau = float(np.float32(32767 / 65536))
    qs = float(np.float32(32767.0 / tau))
    assert qs == 65536.0
    for m, expect in _table("quantize_ties.txt"):
        d = float(np.float32(float(m) / 65536.0))
        assert d == float(m) / 65536.0  # exactly representable
        assert oracle.quantize(d, tau, qs) == int(expect), m


# ---------------------------------------------------------------- ray set-up

def test_ray_setup_geometry():
    """dir is the unit vector sensor->point; int is unit, orthogonal to dir and in
    the plane spanned by dir and up = R e_z (the scan-line normal)."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        R = synth.rot_zyx(*rng.uniform(-math.pi, math.pi, 3))
        t = rng.uniform(-50, 50, 3)
        pose = synth.pose12(R, t)
        p = np.zeros(4, np.float32)
        p[:3] = rng.uniform(-30, 30, 3)
        ry = oracle.ray(pose, p, 0.1, 100.0, 0.01)
        Rf = pose.reshape(3, 4)[:, :3].astype(np.float64)
        v = Rf @ p[:3].astype(np.float64)
        r = np.linalg.norm(v)
        if r < 0.1:
            continue
        assert ry["valid"]
        assert abs(ry["r"] - r) <= 1e-5 * r + 1e-4
        assert np.allclose(ry["dir"], v / r, atol=1e-5)
        up = Rf[:, 2]
        ih = ry["ih"].astype(np.float64)
        assert ry["fill"]
        assert abs(np.linalg.norm(ih) - 1) < 1e-5
        assert abs(ih @ (v / r)) < 1e-5
        assert abs(ih @ np.cross(v / r, up)) < 1e-5


def test_ray_validity():
    pose = synth.pose12(np.eye(3), np.zeros(3))
    assert not oracle.ray(pose, [np.nan, 0, 0, 0], 0.5, 10, 0.01)["valid"]
    assert not oracle.ray(pose, [np.inf, 0, 0, 0], 0.5, 10, 0.01)["valid"]
    assert not oracle.ray(pose, [0, 0, 0, 0], 0.5, 10, 0.01)["valid"]
    assert not oracle.ray(pose, [0.25, 0, 0, 0], 0.5, 10, 0.01)["valid"]
    assert oracle.ray(pose, [0.5, 0, 0, 0], 0.5, 10, 0.01)["valid"]
    assert oracle.ray(pose, [10, 0, 0, 0], 0.5, 10, 0.01)["valid"]
    assert not oracle.ray(pose, [10.5, 0, 0, 0], 0.5, 10, 0.01)["valid"]
    # a ray along up has no interpolation direction
    ry = oracle.ray(pose, [0, 0, 3, 0], 0.5, 10, 0.01)
    assert ry["valid"] and not ry["fill"]
    # delta_z = 0 disables the fill
    assert not oracle.ray(pose, [3, 0, 0, 0], 0.5, 10, 0.0)["fill"]


# ---------------------------------------------------------------- closed-form enumeration

def test_axis_ray_fill_closed_form():
    """The hit list of an axis-aligned ray with fill equals the hand derivation
    in tests/golden/axis_ray_fill.json (Eq. 3 / Eq. 4, int = d x (d x up))."""
    gold = json.load(open(os.path.join(GOLD, "axis_ray_fill.json")))
    p = synth.params_dict(gold["params"]["dims"], gold["params"]["voxel_size"], gold["params"]["tau"],
                          gold["params"]["w_max"], gold["params"]["delta_z"], gold["params"]["r_min"],
                          gold["params"]["r_max"], 0, gold["params"]["origin"])
    assert oracle.derived(p)[2] == gold["K"]
    pts = np.array([gold["point"]], np.float32)
    pose = np.array(gold["pose"], np.float32)
    g, q, _ = oracle.hits(p, pts, pose)
    expect = []
    for s in gold["steps"]:
        for j in range(-s["J"], s["J"] + 1):
            expect.append((s["x"], 0, -j, s["q"]))
    got = [(int(a), int(b), int(c), int(d)) for (a, b, c), d in zip(g, q)]
    assert len(got) == gold["total_hits"]
    assert sorted(got) == sorted(expect)
    # the map after one scan: each voxel hit once, value = its code, weight 1
    m = oracle.OracleMap(p)
    m.integrate(pts, pose)
    v, w = m.read()
    o = p["origin"]
    for x, y, z, code in expect:
        assert v[z - o[2], y - o[1], x - o[0]] == code
        assert w[z - o[2], y - o[1], x - o[0]] == 1
    assert int((w > 0).sum()) == gold["total_hits"]
    assert m.stats() == dict(valid_rays=1, hits=75, touched=75)


def test_no_fill_gives_2k_plus_1_hits():
    """delta_z = 0: every valid ray contributes exactly 2K+1 steps (all in the window)."""
    rng = np.random.default_rng(3)
    p = synth.params_dict((64, 64, 64), 0.1, 0.35, 64, 0.0, 0.5, 2.5, 0, (-32, -32, -32))
    K = oracle.derived(p)[2]
    assert K == 3
    pts = np.zeros((50, 4), np.float32)
    d = rng.normal(size=(50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts[:, :3] = d * rng.uniform(0.8, 2.0, (50, 1))
    pose = synth.pose12(synth.rot_zyx(0.3, 0.1, -0.2), np.array([0.05, -0.1, 0.2]))
    g, q, ray = oracle.hits(p, pts, pose)
    assert len(g) == 50 * (2 * K + 1)
    assert np.all(np.bincount(ray, minlength=50) == 2 * K + 1)


def test_step_distances_follow_ray():
    """Without fill, step k of a ray lands in the voxel containing s + (r + k vs) d
    (FP64 check with a one-voxel tolerance) and its code is within rounding of the
    projective distance of that voxel's centre."""
    rng = np.random.default_rng(4)
    p = synth.params_dict((128, 128, 128), 0.05, 0.2, 64, 0.0, 0.3, 3.0, 0, (-64, -64, -64))
    inv, qs, K = oracle.derived(p)
    pts = np.zeros((40, 4), np.float32)
    d = rng.normal(size=(40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts[:, :3] = d * rng.uniform(0.5, 2.5, (40, 1))
    R = synth.rot_zyx(1.0, 0.2, 0.1)
    t = np.array([0.1, 0.2, -0.3])
    pose = synth.pose12(R, t)
    g, q, ray = oracle.hits(p, pts, pose)
    Rf = pose.reshape(3, 4)[:, :3].astype(np.float64)
    tf = pose.reshape(3, 4)[:, 3].astype(np.float64)
    vs = p["voxel_size"]
    idx = 0
    for i in range(40):
        v = Rf @ pts[i, :3].astype(np.float64)
        r = np.linalg.norm(v)
        dirn = v / r
        for k in range(-K, K + 1):
            l = r + k * vs
            expect_pt = tf + dirn * l
            assert np.all(np.abs((g[idx] + 0.5) * vs - expect_pt) <= 0.5 * vs + 1e-4)
            c = (g[idx] + 0.5) * vs
            dist = r - (c - tf) @ dirn
            dist = min(max(dist, -p["tau"]), p["tau"])
            assert abs(q[idx] - dist * 32767 / p["tau"]) <= 2.0
            idx += 1
    assert idx == len(g)


# ---------------------------------------------------------------- brute force, tiny grids

def _random_scan(rng, n, spread, sensor_box, origin_vox, vs):
    pts = np.zeros((n, 4), np.float32)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts[:, :3] = d * rng.uniform(spread[0], spread[1], (n, 1))
    # a few invalid points
    pts[rng.integers(0, n, max(1, n // 16)), 0] = np.nan
    R = synth.rot_zyx(*rng.uniform(-math.pi, math.pi, 3))
    t = rng.uniform(sensor_box[0], sensor_box[1], 3)
    return pts, synth.pose12(R, t)


@pytest.mark.parametrize("reduce", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_bruteforce_matches_ray_major(reduce, seed):
    """Ray-major oracle == voxel-major brute force (different loop order), bit for
    bit, on 16^3 windows (some straddling negative coordinates) with a random
    pre-existing map, for both per-scan reductions."""
    rng = np.random.default_rng(100 + seed)
    vs = [0.1, 0.125, 0.08][seed % 3]
    origin = [(-8, -8, -8), (0, -16, 8), (-16, 0, -8)][seed % 3]
    tau = [0.2, 0.3, 0.25][seed % 3]
    dz = [0.0, 0.05, 0.2][seed % 3]
    p = synth.params_dict((16, 16, 16), vs, tau, int(rng.integers(1, 20)), dz, 0.05, 3.0, reduce, origin)
    centre = np.array([(o + 8) * vs for o in origin])
    pts, pose = _random_scan(rng, 48, (0.3, 1.0), (centre - 0.2, centre + 0.2), origin, vs)
    v0 = rng.integers(-32767, 32768, size=(16, 16, 16)).astype(np.int16)
    w0 = rng.integers(0, p["w_max"] + 1, size=(16, 16, 16)).astype(np.int16)
    a = oracle.OracleMap(p)
    b = oracle.OracleMap(p)
    a.load_window(v0, w0)
    b.load_window(v0, w0)
    a.integrate(pts, pose)
    b.integrate(pts, pose, bruteforce=True)
    va, wa = a.read()
    vb, wb = b.read()
    assert a.stats()["hits"] > 100
    assert np.array_equal(va, vb) and np.array_equal(wa, wb)
    assert a.stats() == b.stats()


def test_reductions_match_textbook():
    """Per-scan V from the raw contribution list with numpy: WSUM = mean code
    rounded half away from zero, MIN_ABS = code of smallest magnitude (ties to
    the positive value); each applied to an empty map with weight 1 or W."""
    rng = np.random.default_rng(8)
    p0 = synth.params_dict((32, 32, 32), 0.1, 0.3, 1000, 0.05, 0.05, 3.0, 0, (-16, -16, -16))
    p1 = dict(p0, reduce=1)
    pts, pose = _random_scan(rng, 200, (0.4, 1.5), (np.full(3, -0.1), np.full(3, 0.1)), None, 0.1)
    g, q, _ = oracle.hits(p0, pts, pose)
    o = np.array(p0["origin"])
    inside = np.all((g >= o) & (g < o + 32), axis=1)
    g, q = g[inside], q[inside]
    lin = ((g[:, 2] - o[2]) * 32 + (g[:, 1] - o[1])) * 32 + (g[:, 0] - o[0])
    S = np.bincount(lin, weights=q, minlength=32 ** 3).astype(np.int64)
    W = np.bincount(lin, minlength=32 ** 3)
    m0 = oracle.OracleMap(p0)
    m0.integrate(pts, pose)
    v0, w0 = m0.read()
    v0, w0 = v0.reshape(-1), w0.reshape(-1)
    touched = W > 0
    assert np.array_equal(w0, np.minimum(W, 1000).astype(np.int16))
    for i in np.nonzero(touched)[0]:
        x = Fraction(int(S[i]), int(W[i]))
        mag = abs(x)
        e = int(mag + Fraction(1, 2))
        assert v0[i] == (e if x >= 0 else -e)
    # MIN_ABS
    key = np.abs(q).astype(np.int64) * 2 + (q < 0)
    order = np.lexsort((key, lin))
    first = np.ones(len(order), bool)
    first[1:] = lin[order][1:] != lin[order][:-1]
    best = np.zeros(32 ** 3, np.int64)
    best[lin[order][first]] = q[order][first]
    m1 = oracle.OracleMap(p1)
    m1.integrate(pts, pose)
    v1, w1 = m1.read()
    assert np.array_equal(v1.reshape(-1)[touched], best[touched])
    assert np.all(w1.reshape(-1)[touched] == 1) and np.all(w1.reshape(-1)[~touched] == 0)


def test_single_hit_voxels_wsum_equals_min_abs():
    """When every voxel gets at most one contribution, both reductions agree."""
    p = synth.params_dict((64, 64, 64), 0.0625, 0.25, 64, 0.0, 0.1, 5.0, 0, (-32, -32, -32))
    # axis rays with a power-of-two voxel: consecutive steps land in distinct voxels
    pts = np.array([[1.03, 0, 0, 0], [0, -1.52, 0, 0], [0, 0, 1.23, 0]], np.float32)
    pose = synth.pose12(np.eye(3), np.array([0.01, 0.02, 0.03]))
    g, q, _ = oracle.hits(p, pts, pose)
    assert len({tuple(x) for x in g}) == len(g)
    a = oracle.OracleMap(p)
    b = oracle.OracleMap(dict(p, reduce=1))
    a.integrate(pts, pose)
    b.integrate(pts, pose)
    assert all(np.array_equal(x, y) for x, y in zip(a.read(), b.read()))


# ---------------------------------------------------------------- analytic SDF

def _wall_setup(fill):
    vs, tau, sigma = 0.05, 0.2, 0.01
    R = synth.rot_zyx(math.radians(20.0), 0.0, 0.0)
    t = np.array([0.3, -0.2, 0.1])
    d_wall = 3.0 - t[0]
    r_max = d_wall / math.cos(math.radians(20.0))
    scene = synth.Scene(boxes=np.array([[3.0, -50.0, -50.0, 10.0, 50.0, 50.0]]))
    dirs = synth.beam_directions(16, 360, -15.0, 15.0)
    pts = synth.make_scan(scene, R, t, dirs, sigma, synth.SplitMix64(77), r_max=r_max)
    dz = synth.delta_z_for(30.0, 16) if fill else 0.0
    p = synth.params_dict((128, 128, 64), vs, tau, 64, dz, 0.3, r_max, 0, (-64, -64, -32))
    return p, pts, synth.pose12(R, t), sigma, r_max


@pytest.mark.parametrize("fill", [False, True])
def test_planar_wall_sdf(fill):
    """Wall x = 3 m seen at incidence <= 20 deg from a rotated, translated sensor:
    every observed voxel satisfies |tau v / QMAX - clamp(3 - c_x)| <= vs + 3 sigma
    (+ h_max sin 15 deg with fill), against the FP64 signed distance."""
    p, pts, pose, sigma, r_max = _wall_setup(fill)
    m = oracle.OracleMap(p)
    m.integrate(pts, pose)
    v, w = m.read()
    st = m.stats()
    assert st["valid_rays"] > 300 and st["touched"] > 1000
    zz, yy, xx = np.nonzero(w > 0)
    o = p["origin"]
    vs = p["voxel_size"]
    cx = (xx + o[0] + 0.5) * vs
    sdf = np.clip(3.0 - cx, -p["tau"], p["tau"])
    val = v[zz, yy, xx].astype(np.float64) * p["tau"] / 32767.0
    bound = vs + 3 * sigma
    if fill:
        h_max = p["delta_z"] * (r_max + p["tau"])
        bound += h_max * math.sin(math.radians(15.0))
    err = np.abs(val - sdf)
    assert err.max() <= bound, (err.max(), bound)
    # the sign convention: positive in front of the surface (sensor side)
    assert np.all(val[cx < 3.0 - vs - 3 * sigma - 0.03] > 0)
    assert np.all(val[cx > 3.0 + vs + 3 * sigma + 0.03] < 0)


def test_planar_wall_catches_transposed_rotation():
    """Mutation check: the same scan with R transposed (a plausible mistake)
    violates the wall bound, so the bound above does pin the transform."""
    p, pts, pose, sigma, r_max = _wall_setup(False)
    M = pose.reshape(3, 4).copy()
    M[:, :3] = M[:, :3].T
    m = oracle.OracleMap(p)
    m.integrate(pts, M.reshape(12))
    v, w = m.read()
    zz, yy, xx = np.nonzero(w > 0)
    cx = (xx + p["origin"][0] + 0.5) * p["voxel_size"]
    val = v[zz, yy, xx] * p["tau"] / 32767.0
    err = np.abs(val - np.clip(3.0 - cx, -p["tau"], p["tau"]))
    assert err.max() > p["voxel_size"] + 3 * sigma


def test_box_room_accuracy():
    """Box room (16 x 360 beams, 0.05 m voxels, tau 0.2): most observed voxels are
    within vs + 3 sigma (+ fill height) of the FP64 signed distance of room + box."""
    w = synth.workload_room()
    p = w.params
    m = oracle.OracleMap(p)
    m.integrate(w.scans[0], w.poses[0])
    v, wt = m.read()
    zz, yy, xx = np.nonzero(wt > 0)
    o = p["origin"]
    vs = p["voxel_size"]
    c = np.stack([(xx + o[0] + 0.5) * vs, (yy + o[1] + 0.5) * vs, (zz + o[2] + 0.5) * vs], axis=1)
    ud = w.scene.sdf(c)
    room = w.scene.room
    inside_room = np.all((c > room[:3]) & (c < room[3:]), axis=1)
    bx = w.scene.boxes[0]
    in_box = np.all((c > bx[:3]) & (c < bx[3:]), axis=1)
    sdf = np.where(inside_room & ~in_box, ud, -ud)
    sdf = np.clip(sdf, -p["tau"], p["tau"])
    val = v[zz, yy, xx] * p["tau"] / 32767.0
    h_max = p["delta_z"] * 8.0
    ok = np.abs(val - sdf) <= vs + 0.03 + h_max * math.sin(math.radians(15))
    assert ok.mean() > 0.9, ok.mean()
    assert m.stats()["valid_rays"] == 5760


# ---------------------------------------------------------------- invariants

def test_invariants_room_scan():
    w = synth.workload_room()
    p = w.params
    rng = np.random.default_rng(9)
    dims = p["dims"]
    v0 = rng.integers(-32767, 32768, size=(dims[2], dims[1], dims[0])).astype(np.int16)
    w0 = rng.integers(0, 65, size=v0.shape).astype(np.int16)
    m = oracle.OracleMap(p)
    m.load_window(v0, w0)
    m.integrate(w.scans[0], w.poses[0])
    v1, w1 = m.read()
    # weight never exceeds Wmax; untouched voxels are byte-identical
    assert w1.max() <= p["w_max"]
    g, q, _ = oracle.hits(p, w.scans[0], w.poses[0])
    o = np.array(p["origin"])
    inside = np.all((g >= o) & (g < o + np.array(dims)), axis=1)
    g = g[inside] - o
    touched = np.zeros(v0.shape, bool)
    touched[g[:, 2], g[:, 1], g[:, 0]] = True
    assert np.array_equal(v1[~touched], v0[~touched]) and np.array_equal(w1[~touched], w0[~touched])
    assert np.all(w1[touched] >= np.minimum(w0[touched] + 1, p["w_max"]))
    assert m.stats()["touched"] == int(touched.sum())
    assert m.stats()["hits"] == int(inside.sum())


def test_same_scan_twice():
    """Integrating one scan twice into an empty map: value moves by at most one
    code, weight doubles (clamped)."""
    w = synth.workload_room()
    m = oracle.OracleMap(w.params)
    m.integrate(w.scans[0], w.poses[0])
    v1, w1 = m.read()
    m.integrate(w.scans[0], w.poses[0])
    v2, w2 = m.read()
    t = w1 > 0
    assert np.abs(v2[t].astype(np.int32) - v1[t]).max() <= 1
    assert np.array_equal(w2[t], np.minimum(2 * w1[t].astype(np.int32), w.params["w_max"]).astype(np.int16))
    assert np.array_equal(w2[~t], w1[~t])


def test_empty_and_invalid_scans():
    w = synth.workload_room()
    m = oracle.OracleMap(w.params)
    m.integrate(np.zeros((0, 4), np.float32), w.poses[0])
    assert m.stats() == dict(valid_rays=0, hits=0, touched=0)
    bad = np.full((100, 4), np.nan, np.float32)
    bad[:50] = 0.0
    m.integrate(bad, w.poses[0])
    v, wt = m.read()
    assert m.stats() == dict(valid_rays=0, hits=0, touched=0)
    assert not v.any() and not wt.any()


# ---------------------------------------------------------------- shift

def _map_after_room_scan(shift_dims=(128, 128, 64)):
    w = synth.workload_room()
    p = dict(w.params, dims=shift_dims, origin=synth.window_origin((0, 0, 0), shift_dims, 0.05))
    m = oracle.OracleMap(p)
    m.integrate(w.scans[0], w.poses[0])
    return m, p, w


def test_shift_zero_is_noop():
    m, p, _ = _map_after_room_scan()
    v0, w0 = m.read()
    m.shift(p["origin"])
    v1, w1 = m.read()
    assert np.array_equal(v0, v1) and np.array_equal(w0, w1)


@pytest.mark.parametrize("delta", [(8, 0, 0), (-16, 8, 0), (0, 0, 8), (24, -40, 16), (200, 0, 0)])
def test_shift_then_unshift_identity(delta):
    m, p, _ = _map_after_room_scan()
    o = p["origin"]
    v0, w0 = m.read()
    assert w0.any()
    no = tuple(o[a] + delta[a] for a in range(3))
    m.shift(no)
    assert m.origin == no
    m.shift(o)
    v1, w1 = m.read()
    assert np.array_equal(v0, v1) and np.array_equal(w0, w1)


def test_shift_preserves_global_coordinates():
    """A voxel keeps its value (read by global coordinates) while it stays in the
    window; voxels that enter for the first time are (0, 0)."""
    m, p, _ = _map_after_room_scan()
    o = np.array(p["origin"])
    d = np.array(p["dims"])
    delta = np.array([16, -8, 8])
    no = o + delta
    lo = np.maximum(o, no)
    hi = np.minimum(o + d, no + d)
    before = m.read(tuple(lo), tuple(hi))
    m.shift(tuple(no))
    after = m.read(tuple(lo), tuple(hi))
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    v, w = m.read()
    # region x >= o.x + d.x (relative to the new origin) is new
    new_x0 = int(o[0] + d[0] - no[0])
    assert not v[:, :, new_x0:].any() and not w[:, :, new_x0:].any()


def test_shift_store_drops_empty_chunks():
    m, p, _ = _map_after_room_scan()
    o = p["origin"]
    m.shift((o[0] + 512, o[1], o[2]))   # everything leaves
    v, w = m.read()
    assert not v.any() and not w.any()
    n_store = m.store_chunks()
    assert 0 < n_store < (128 * 128 * 64) // 512   # only non-empty chunks were kept
    m.shift(o)
    v1, w1 = m.read()
    assert w1.any()


def test_shift_rejects_unaligned_origin():
    m, p, _ = _map_after_room_scan()
    with pytest.raises(ValueError):
        m.shift((p["origin"][0] + 3, p["origin"][1], p["origin"][2]))


def test_integrate_after_shift_matches_bigger_window():
    """Integrating into a shifted window gives the same values as integrating
    into a window that never moved and covers the same voxels."""
    w = synth.workload_room()
    dims_small = (64, 64, 32)
    o_small = (-32, -32, -16)
    ps = dict(w.params, dims=dims_small, origin=o_small)
    m = oracle.OracleMap(ps)
    m.shift((-24, -40, -16))
    m.integrate(w.scans[0], w.poses[0])
    big = oracle.OracleMap(dict(w.params, dims=(128, 128, 64), origin=(-64, -64, -32)))
    big.integrate(w.scans[0], w.poses[0])
    a = m.read()
    b = big.read((-24, -40, -16), (40, 24, 16))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ---------------------------------------------------------------- alternative readings (map flags)

FLAG_STEP, FLAG_SCAN = 1, 2


def test_eq12_scan_weight_golden_table():
    """Eq. 1 / Eq. 2 with the scan's average as one observation, against the
    hand-computed table (tests/golden/eq12_scan_table.txt)."""
    rows = _table("eq12_scan_table.txt")
    assert len(rows) >= 15
    for r in rows:
        gv, gw, S, W, wmax, ev, ew = (int(x) for x in r)
        assert oracle.eq12(gv, gw, S, W, wmax, scan_weight=True) == (ev, ew), r


def test_eq12_scan_weight_exact_rational():
    """Random cases against exact rationals: value = (gv*gw + S/W)/(gw+1) rounded
    half away from zero; with W = 1 it is plain Eq. 1."""
    rng = np.random.default_rng(15)
    for _ in range(3000):
        gv = int(rng.integers(-32767, 32768))
        gw = int(rng.integers(0, 65))
        W = int(rng.integers(1, 300))
        S = int(rng.integers(-32767, 32768)) * W // max(1, int(rng.integers(1, 4)))
        wmax = int(rng.integers(1, 65))
        x = (Fraction(gv * gw) + Fraction(S, W)) / (gw + 1)
        mag = math.floor(abs(x) + Fraction(1, 2))
        ev = mag if x >= 0 else -mag
        assert oracle.eq12(gv, gw, S, W, wmax, scan_weight=True) == (ev, min(wmax, gw + 1))
        if W == 1:
            assert oracle.eq12(gv, gw, S, 1, wmax, scan_weight=True) == oracle.eq12(gv, gw, S, 1, wmax)


def test_step_value_closed_form():
    """Step-valued fill: every voxel of march step k, the ray voxel and all its
    vertical fill voxels, carries the code of d = r - l = -k * voxel. With
    r = 1.5, voxel 0.125 and tau 0.5 all of it is exact in binary32, so the
    codes are rint(-k * 0.125 * 65534), ties to even:
    k = -4..4 -> 32767, 24575, 16384, 8192, 0, -8192, -16384, -24575, -32767."""
    expect = {-4: 32767, -3: 24575, -2: 16384, -1: 8192, 0: 0, 1: -8192, 2: -16384, 3: -24575, 4: -32767}
    pose = synth.pose12(np.eye(3), np.array([0.25, -0.5, 0.125]))
    pts = np.array([[0.5, 1.0, 1.0, 0.0]], np.float32)          # |p| = 1.5 exactly, oblique
    for dz in (0.0, 0.1):
        p = synth.params_dict((64, 64, 64), 0.125, 0.5, 64, dz, 0.1, 10.0, 0, (-32, -32, -32),
                              flags=FLAG_STEP)
        assert oracle.derived(p)[1] == np.float32(65534.0)
        g, q, _, k = oracle.hits(p, pts, pose, with_k=True)
        assert sorted(set(k.tolist())) == list(range(-4, 5))
        for kk, qq in zip(k.tolist(), q.tolist()):
            assert qq == expect[kk]
        counts = np.bincount(k + 4)
        if dz == 0.0:
            assert np.all(counts == 1)
        else:
            # J = floor(0.1 * l / 0.125) per side at l = 1.5 + 0.125 k
            J = [math.floor(0.1 * (1.5 + 0.125 * kk) / 0.125) for kk in range(-4, 5)]
            assert counts.tolist() == [2 * j + 1 for j in J]
        # the default projective reading differs off the ray's voxel centres
        p0 = dict(p, flags=0)
        _, q0, _ = oracle.hits(p0, pts, pose)
        assert len(q0) == len(q) and not np.array_equal(q0, q)


def test_step_value_vs_projective_on_axis():
    """On an axis-aligned ray through voxel centres, the step's distance and the
    projective distance of the ray voxel coincide: the codes of the j = 0 voxels
    agree between the two readings (tests/golden/axis_ray_fill.json geometry)."""
    gold = json.load(open(os.path.join(GOLD, "axis_ray_fill.json")))
    gp = gold["params"]
    p = synth.params_dict(gp["dims"], gp["voxel_size"], gp["tau"], gp["w_max"], gp["delta_z"], gp["r_min"],
                          gp["r_max"], 0, gp["origin"])
    pts = np.array([gold["point"]], np.float32)
    pose = np.array(gold["pose"], np.float32)
    g0, q0, _, k0 = oracle.hits(p, pts, pose, with_k=True)
    g1, q1, _, k1 = oracle.hits(dict(p, flags=FLAG_STEP), pts, pose, with_k=True)
    assert np.array_equal(g0, g1) and np.array_equal(k0, k1)
    steps = {s["x"]: s["q"] for s in gold["steps"]}
    for (x, y, z), qa, qb in zip(g0.tolist(), q0.tolist(), q1.tolist()):
        assert qb == steps[x]            # every voxel of a step takes the step's code
        if z == 0:
            assert qa == qb


@pytest.mark.parametrize("flags", [FLAG_STEP, FLAG_SCAN, FLAG_STEP | FLAG_SCAN])
@pytest.mark.parametrize("reduce", [0, 1])
@pytest.mark.parametrize("seed", range(3))
def test_bruteforce_matches_ray_major_flags(flags, reduce, seed):
    """Both readings through the voxel-major brute force, bit for bit."""
    rng = np.random.default_rng(300 + seed)
    vs = [0.1, 0.125, 0.08][seed]
    origin = [(-8, -8, -8), (0, -16, 8), (-16, 0, -8)][seed]
    p = synth.params_dict((16, 16, 16), vs, [0.2, 0.3, 0.25][seed], int(rng.integers(1, 20)),
                          [0.05, 0.2, 0.1][seed], 0.05, 3.0, reduce, origin, flags=flags)
    centre = np.array([(o + 8) * vs for o in origin])
    pts, pose = _random_scan(rng, 48, (0.3, 1.0), (centre - 0.2, centre + 0.2), origin, vs)
    v0 = rng.integers(-32767, 32768, size=(16, 16, 16)).astype(np.int16)
    w0 = rng.integers(0, p["w_max"] + 1, size=(16, 16, 16)).astype(np.int16)
    a, b = oracle.OracleMap(p), oracle.OracleMap(p)
    a.load_window(v0, w0)
    b.load_window(v0, w0)
    a.integrate(pts, pose)
    b.integrate(pts, pose, bruteforce=True)
    assert a.stats()["hits"] > 100
    va, wa = a.read()
    vb, wb = b.read()
    assert np.array_equal(va, vb) and np.array_equal(wa, wb)


def test_scan_weight_relations():
    """Per-scan weight reading on a room scan: on an empty map the values equal
    the default reading's and every touched weight is 1; a second identical
    scan leaves values within one code and raises each weight by exactly 1;
    MIN_ABS (weight 1 per scan already) is unchanged by the flag."""
    w = synth.workload_room(seed=9)
    pts, pose, p = w.scans[0], w.poses[0], w.params
    base = oracle.OracleMap(p)
    scan = oracle.OracleMap(dict(p, flags=FLAG_SCAN))
    base.integrate(pts, pose)
    scan.integrate(pts, pose)
    vb, wb = base.read()
    vs_, ws = scan.read()
    assert np.array_equal(vb, vs_)
    assert np.array_equal(ws, (wb > 0).astype(np.int16))
    assert int(wb.max()) > 1
    scan.integrate(pts, pose)
    v2, w2 = scan.read()
    t = ws > 0
    assert np.all(np.abs(v2[t].astype(int) - vs_[t].astype(int)) <= 1)
    assert np.array_equal(w2[t], np.minimum(ws[t] + 1, p["w_max"]))
    for fl in (0, FLAG_SCAN):
        m = oracle.OracleMap(dict(p, reduce=1, flags=fl))
        m.integrate(pts, pose)
        if fl == 0:
            ref = m.read()
        else:
            got = m.read()
            assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])


def test_oracle_rejects_unknown_flag_bits():
    p = synth.params_dict((16, 16, 16), 0.1, 0.2, 8, 0.0, 0.05, 3.0, 0, (0, 0, 0), flags=4)
    with pytest.raises(ValueError):
        oracle.OracleMap(p)


# ---------------------------------------------------------------- zero-crossing surface (map consumer)

def _surface_map(v, w, vs=0.25):
    Z, Y, X = v.shape
    p = synth.params_dict((X, Y, Z), vs, 4 * vs, 64, 0.0, 0.1, 10.0, 0, (0, 0, 0))
    m = oracle.OracleMap(p)
    m.load_window(v.astype(np.int16), w.astype(np.int16))
    return m


def _sign_changes(v, w, min_w):
    """Numpy brute force: crossings per axis (x, y, z) of a (z, y, x) field."""
    ok = w >= min_w
    neg = v < 0
    out = []
    for ax, sl_a, sl_b in ((0, np.s_[:, :, :-1], np.s_[:, :, 1:]), (1, np.s_[:, :-1, :], np.s_[:, 1:, :]),
                           (2, np.s_[:-1, :, :], np.s_[1:, :, :])):
        out.append(int(np.sum(ok[sl_a] & ok[sl_b] & (neg[sl_a] != neg[sl_b]))))
    return out


def test_surface_axis_plane_closed_form():
    """A field linear in x with its zero at x = 7.3 voxels gives one point per
    (y, z) row at exactly ((6 + 0.5) + 0.8) * 0.25 = 1.825 m."""
    xs = np.arange(16)
    v = np.broadcast_to(np.rint(1000 * (xs + 0.5 - 7.3)), (16, 16, 16)).astype(np.int16)
    m = _surface_map(v, np.ones_like(v))
    pts = m.surface()
    assert pts.shape == (256, 4)
    assert np.all(pts[:, 3] == 0)
    assert np.all(np.abs(pts[:, 0] - 1.825) < 1e-6)
    assert sorted(set(np.round(pts[:, 1] / 0.25 - 0.5).astype(int))) == list(range(16))


@pytest.mark.parametrize("seed", range(4))
def test_surface_tilted_plane_and_counts(seed):
    """A linear field of a tilted plane: every point lies on the plane within
    the rounding of the codes, and the number of points per axis equals a
    numpy count of sign changes between observed neighbours."""
    rng = np.random.default_rng(40 + seed)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    c0 = rng.uniform(6, 10, 3)
    s = 1000.0
    zz, yy, xx = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    cen = np.stack([xx + 0.5, yy + 0.5, zz + 0.5], axis=-1)
    v = np.rint(s * ((cen - c0) @ n)).clip(-32767, 32767).astype(np.int16)
    w = (rng.uniform(size=v.shape) < 0.8).astype(np.int16) * rng.integers(1, 5, size=v.shape).astype(np.int16)
    for min_w in (1, 3):
        m = _surface_map(v, w, vs=0.25)
        pts = m.surface(min_w)
        per_axis = [int(np.sum(pts[:, 3] == a)) for a in range(3)]
        assert per_axis == _sign_changes(v, w, min_w)
        d = (pts[:, :3].astype(np.float64) / 0.25 - c0) @ n
        ax = pts[:, 3].astype(int)
        tol = 0.5 / (s * np.abs(n[ax])) + 1e-4
        assert np.all(np.abs(d) <= tol)


def test_surface_of_room_scan_near_walls():
    """Points extracted from the box-room scan lie near the room's surfaces
    (FP64 analytic distance, one voxel + 3 sigma)."""
    w = synth.workload_room(seed=3)
    m = oracle.OracleMap(w.params)
    m.integrate(w.scans[0], w.poses[0])
    pts = m.surface(1)
    assert len(pts) > 10000
    dist = np.abs(w.scene.sdf(pts[:, :3].astype(np.float64)))
    assert np.mean(dist <= w.params["voxel_size"] + 0.03) > 0.95


# ---------------------------------------------------------------- parallel oracle (host-core timing)

@pytest.mark.parametrize("reduce", [0, 1])
def test_parallel_oracle_identical(reduce):
    """The ray-split, multithreaded oracle merges integer per-scan volumes, so
    it equals the serial oracle bit for bit (with a pre-filled window)."""
    w = synth.workload_room(reduce=reduce, seed=6)
    rng = np.random.default_rng(7)
    d = w.params["dims"]
    v0 = rng.integers(-32767, 32768, size=(d[2], d[1], d[0])).astype(np.int16)
    w0 = rng.integers(0, 65, size=v0.shape).astype(np.int16)
    a, b = oracle.OracleMap(w.params), oracle.OracleMap(w.params)
    a.load_window(v0, w0)
    b.load_window(v0, w0)
    a.integrate(w.scans[0], w.poses[0])
    b.integrate(w.scans[0], w.poses[0], threads=5)
    va, wa = a.read()
    vb, wb = b.read()
    assert np.array_equal(va, vb) and np.array_equal(wa, wb)
    assert a.stats() == b.stats()


# ---------------------------------------------------------------- scan-to-map registration (map consumer)

def _box_sdf_map(vs=0.05, tau=0.2, half=(0.6, 0.4, 0.3), rot=(0.3, 0.2, 0.1)):
    """A 64^3 window holding the exact (truncated, quantised) signed distance
    of a rotated box, every voxel observed."""
    p = synth.params_dict((64, 64, 64), vs, tau, 64, 0.0, 0.1, 10.0, 0, (-32, -32, -32))
    Rb = synth.rot_zyx(*rot)
    half = np.array(half)
    g = np.stack(np.meshgrid(np.arange(-32, 32), np.arange(-32, 32), np.arange(-32, 32), indexing="ij"), -1)
    cen = (g[..., ::-1] + 0.5) * vs
    qd = np.abs(cen @ Rb) - half
    sdf = np.linalg.norm(np.maximum(qd, 0), axis=-1) + np.minimum(qd.max(-1), 0)
    v = np.rint(np.clip(sdf, -tau, tau) * 32767 / tau).astype(np.int16)
    m = oracle.OracleMap(p)
    m.load_window(v, np.ones_like(v))
    rng = np.random.default_rng(0)
    n = 4000
    face = rng.integers(0, 6, n)
    u = rng.uniform(-1, 1, (n, 3)) * half
    ax = face % 3
    u[np.arange(n), ax] = np.where(face < 3, 1.0, -1.0) * half[ax]
    pts = np.zeros((n, 4), np.float32)
    pts[:, :3] = u @ Rb.T
    return m, p, pts


def test_register_system_linear_field_closed_form():
    """A field linear in x (code 100 (g_x - 10)) is interpolated exactly: with
    the identity pose each point's residual is (tau/32767) 100 (u_x - 10) with
    u = x / vs - 0.5 in binary32, its gradient (tau/32767) 100 / vs e_x, and
    H, g, cost and count follow in closed form."""
    vs, tau = 0.1, 0.3
    p = synth.params_dict((32, 32, 32), vs, tau, 64, 0.0, 0.1, 10.0, 0, (0, 0, 0))
    xs = np.arange(32)
    v = np.broadcast_to(100 * (xs - 10), (32, 32, 32)).astype(np.int16)
    m = oracle.OracleMap(p)
    m.load_window(v, np.ones_like(v))
    rng = np.random.default_rng(1)
    pts = np.zeros((300, 4), np.float32)
    pts[:, :3] = rng.uniform(0.2, 3.0, (300, 3)).astype(np.float32)
    pose = synth.pose12(np.eye(3), np.zeros(3))
    sysv = m.register_system(pts, pose)
    inv = oracle.derived(p)[0]
    u = (pts[:, 0] * np.float32(inv)) - np.float32(0.5)
    scale = np.float64(np.float32(tau)) / 32767
    d = scale * 100 * (u.astype(np.float64) - 10)
    gr = np.array([scale * 100 / np.float64(np.float32(vs)), 0.0, 0.0])
    q = pts[:, :3].astype(np.float64)
    J = np.concatenate([np.cross(q, gr), np.broadcast_to(gr, q.shape)], axis=1)
    H = J.T @ J
    assert sysv[28] == 300
    assert np.isclose(sysv[27], np.sum(d * d), rtol=1e-12)
    assert np.allclose(sysv[21:27], J.T @ d, rtol=1e-10, atol=1e-15)
    assert np.allclose(sysv[:21], H[np.triu_indices(6)], rtol=1e-10, atol=1e-15)


def test_register_jacobian_matches_finite_differences():
    """g = sum J r is half the derivative of the cost along each pose
    direction (w: rotation about the origin, v: translation), checked with
    central differences of the cost on an exact box field."""
    m, p, pts = _box_sdf_map()
    base = synth.pose12(synth.rot_zyx(0.01, -0.008, 0.006), np.array([0.01, -0.012, 0.008]))
    sysv = m.register_system(pts, base)
    P = base.reshape(3, 4).astype(np.float64)
    eps = 2e-4
    for k in range(6):
        costs = []
        for sgn in (1, -1):
            xi = np.zeros(6)
            xi[k] = sgn * eps
            w, vv = xi[:3], xi[3:]
            K = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
            E = np.eye(3) + K + 0.5 * K @ K
            Q = np.concatenate([E @ P[:, :3], (E @ P[:, 3] + vv)[:, None]], axis=1).astype(np.float32).reshape(12)
            costs.append(m.register_system(pts, Q)[27])
        fd = (costs[0] - costs[1]) / (2 * eps)
        assert abs(fd - 2 * sysv[21 + k]) <= 0.02 * abs(2 * sysv[21 + k]) + 1e-6, (k, fd, 2 * sysv[21 + k])


def test_register_recovers_box_pose():
    """Gauss-Newton on an exact box field recovers a pose perturbed by about
    1 degree and 4 cm to within 0.5 mm and 0.1 degree."""
    m, p, pts = _box_sdf_map()
    pose = synth.pose12(synth.rot_zyx(np.deg2rad(1.0), np.deg2rad(-0.7), np.deg2rad(0.5)),
                        np.array([0.03, -0.02, 0.025]))
    for _ in range(6):
        pose, xi = oracle.pose_update(pose, m.register_system(pts, pose))
    P = pose.reshape(3, 4).astype(np.float64)
    ang = np.rad2deg(np.arccos(np.clip((np.trace(P[:, :3]) - 1) / 2, -1, 1)))
    assert np.linalg.norm(P[:, 3]) < 5e-4 and ang < 0.1
    assert np.linalg.norm(xi) < 1e-4


# ---------------------------------------------------------------- marching-tetrahedra mesh (map consumer)

def _sphere_map(r=0.55, c0=(0.03, -0.02, 0.05), vs=0.05, tau=0.2):
    p = synth.params_dict((48, 48, 48), vs, tau, 64, 0.0, 0.1, 10.0, 0, (-24, -24, -24))
    g = np.stack(np.meshgrid(np.arange(-24, 24), np.arange(-24, 24), np.arange(-24, 24), indexing="ij"), -1)
    cen = (g[..., ::-1] + 0.5) * vs
    sdf = np.linalg.norm(cen - np.array(c0), axis=-1) - r
    v = np.rint(np.clip(sdf, -tau, tau) * 32767 / tau).astype(np.int16)
    m = oracle.OracleMap(p)
    m.load_window(v, np.ones_like(v))
    return m, np.array(c0), r


def test_mesh_plane_area_and_orientation_closed_form():
    """A field linear in x with its zero at 7.3 voxels: the mesh is the plane
    x = 1.825 m across the 15 x 15 dual cells (area 225 * 0.25^2), every
    normal along +x (towards positive distance)."""
    xs = np.arange(16)
    v = np.broadcast_to(np.rint(1000 * (xs + 0.5 - 7.3)), (16, 16, 16)).astype(np.int16)
    m = _surface_map(v, np.ones_like(v))
    tri = m.mesh().astype(np.float64)
    assert np.all(np.abs(tri[:, :, 0] - 1.825) < 1e-6)
    nrm = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    assert np.all(nrm[:, 0] > 0)
    assert np.isclose(0.5 * np.linalg.norm(nrm, axis=1).sum(), 225 * 0.0625, rtol=1e-5)


def test_mesh_sphere_is_closed_oriented_manifold():
    """A sphere inside the window: every edge of the mesh is shared by exactly
    two triangles with opposite directions (closed, consistently oriented
    2-manifold), V - E + F = 2, normals point outwards, and the vertices lie
    within a small fraction of a voxel of the sphere."""
    m, c0, r = _sphere_map()
    tri = m.mesh()
    assert len(tri) > 1000
    keys = {}
    verts = tri.reshape(-1, 3)
    vid = np.unique(verts, axis=0, return_inverse=True)[1].reshape(-1, 3)
    edges = {}
    for t in vid:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            edges.setdefault((min(a, b), max(a, b)), []).append((a, b))
    assert all(len(e) == 2 and e[0] != e[1] for e in edges.values())
    V, E, F = vid.max() + 1, len(edges), len(vid)
    assert V - E + F == 2
    t64 = tri.astype(np.float64)
    nrm = np.cross(t64[:, 1] - t64[:, 0], t64[:, 2] - t64[:, 0])
    cent = t64.mean(axis=1)
    assert np.all(np.einsum("ij,ij->i", nrm, cent - c0) > 0)
    assert np.all(np.abs(np.linalg.norm(verts.astype(np.float64) - c0, axis=1) - r) < 0.15 * 0.05)


def test_mesh_of_room_map_near_walls():
    """The mesh of a scanned room lies near the room's surfaces (FP64 analytic
    distance, one voxel + 3 sigma, for 90 % of the vertices)."""
    w = synth.workload_room(seed=3)
    m = oracle.OracleMap(w.params)
    m.integrate(w.scans[0], w.poses[0])
    tri = m.mesh()
    assert len(tri) > 1000
    dist = np.abs(w.scene.sdf(tri.reshape(-1, 3).astype(np.float64)))
    assert np.mean(dist <= w.params["voxel_size"] + 0.03) > 0.9
