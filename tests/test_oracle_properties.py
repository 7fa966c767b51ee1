"""Property tests of the oracle (hypothesis): Eq. 1 / Eq. 2 identities, the
quantiser, ray set-up invariants, the shift as a permutation of the global
map, and order independence of a scan. Each property is a fact of the
mathematics or of the method, checked on generated inputs."""
import math
from fractions import Fraction

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
from paper_2310_05766_gb300 import synth  # noqa: E402

code = st.integers(-32767, 32767)
weight = st.integers(0, 32767)


@settings(max_examples=400, deadline=None)
@given(gv=code, gw=weight, q=code, wmax=st.integers(1, 32767))
def test_eq12_single_observation_properties(gv, gw, q, wmax):
    """One contribution (S = q, W = 1): the new value lies between the old
    value and q (a convex combination, up to the final rounding), the weight
    is min(wmax, gw + 1), and an empty voxel takes q exactly."""
    gw = min(gw, wmax)
    nv, nw = oracle.eq12(gv, gw, q, 1, wmax)
    assert nw == min(wmax, gw + 1)
    assert min(gv, q) <= nv <= max(gv, q)
    if gw == 0:
        assert nv == q
    exact = Fraction(gv * gw + q, gw + 1)
    assert abs(nv - exact) <= Fraction(1, 2)


@settings(max_examples=300, deadline=None)
@given(gv=code, gw=st.integers(0, 64), S=st.integers(-32767 * 50, 32767 * 50), W=st.integers(1, 50),
       wmax=st.integers(1, 64))
def test_eq12_matches_exact_rational(gv, gw, S, W, wmax):
    gw = min(gw, wmax)
    S = max(-32767 * W, min(32767 * W, S))        # a sum of W codes
    nv, nw = oracle.eq12(gv, gw, S, W, wmax)
    x = Fraction(gv * gw + S, gw + W)
    mag = math.floor(abs(x) + Fraction(1, 2))
    assert nv == (mag if x >= 0 else -mag)
    assert nw == min(wmax, gw + W)
    assert abs(nv) <= 32767


@settings(max_examples=300, deadline=None)
@given(gv=code, gw=st.integers(0, 64), S=st.integers(-32767 * 20, 32767 * 20), W=st.integers(1, 20))
def test_scan_weight_reading_is_eq12_of_the_mean(gv, gw, S, W):
    """The one-observation-per-scan reading equals Eq. 1 with the scan's mean
    code as a single observation, computed as an exact rational."""
    S = max(-32767 * W, min(32767 * W, S))
    nv, nw = oracle.eq12(gv, gw, S, W, 64, scan_weight=True)
    x = (Fraction(gv * gw) + Fraction(S, W)) / (gw + 1)
    mag = math.floor(abs(x) + Fraction(1, 2))
    assert nv == (mag if x >= 0 else -mag) and nw == min(64, gw + 1)


@settings(max_examples=300, deadline=None)
@given(a=st.floats(-1.0, 1.0, width=32), b=st.floats(-1.0, 1.0, width=32), tau=st.sampled_from([0.1, 0.2, 0.6]))
def test_quantiser_monotone_odd_and_clamped(a, b, tau):
    qs = oracle.derived(synth.params_dict((8, 8, 8), tau / 4, tau, 8, 0.0, 0.1, 10.0))[1]
    qa, qb = oracle.quantize(a, np.float32(tau), qs), oracle.quantize(b, np.float32(tau), qs)
    if a <= b:
        assert qa <= qb
    assert oracle.quantize(-a, np.float32(tau), qs) == -qa       # ties to even are symmetric
    assert abs(qa) <= 32767
    if abs(a) >= tau:
        assert abs(qa) == 32767


@settings(max_examples=200, deadline=None)
@given(x=st.floats(-30, 30), y=st.floats(-30, 30), z=st.floats(-5, 5), yaw=st.floats(-3.1, 3.1),
       roll=st.floats(-0.3, 0.3))
def test_ray_setup_invariants(x, y, z, yaw, roll):
    """A valid ray has a unit direction along the point, and its fill
    direction is a unit vector orthogonal to it (int = d x (d x up))."""
    pose = synth.pose12(synth.rot_zyx(yaw, 0.1, roll), np.array([0.5, -0.2, 0.3]))
    r = oracle.ray(pose, [x, y, z, 0.0], 0.3, 100.0, 0.01)
    rng = math.sqrt(x * x + y * y + z * z)
    if not (0.3 <= rng <= 100.0) or rng < 0.31 or rng > 99.9:
        return
    assert r["valid"]
    d = r["dir"].astype(np.float64)
    assert abs(np.linalg.norm(d) - 1) < 1e-5
    assert abs(r["r"] - rng) < 1e-4 * max(1.0, rng)
    if r["fill"]:
        ih = r["ih"].astype(np.float64)
        assert abs(np.linalg.norm(ih) - 1) < 1e-5
        assert abs(ih @ d) < 1e-4


_ROOM = None


def _room():
    global _ROOM
    if _ROOM is None:
        w = synth.workload_room(seed=12)
        _ROOM = (dict(w.params, dims=(64, 64, 32), origin=(-32, -32, -16), voxel_size=0.1), w.scans[0], w.poses[0])
    return _ROOM


@settings(max_examples=25, deadline=None)
@given(moves=st.lists(st.tuples(st.integers(-6, 6), st.integers(-6, 6), st.integers(-3, 3)), min_size=1, max_size=4))
def test_shifts_preserve_the_global_map(moves):
    """Any sequence of shifts only moves chunks between the window and the
    store; shifting back to the start restores the window exactly."""
    p, pts, pose = _room()
    m = oracle.OracleMap(p)
    m.integrate(pts, pose)
    ref = m.global_chunks()
    v0, w0 = m.read()
    o = list(p["origin"])
    for dx, dy, dz in moves:
        o = [o[0] + 8 * dx, o[1] + 8 * dy, o[2] + 8 * dz]
        m.shift(tuple(o))
    got = m.global_chunks()
    assert got.keys() == ref.keys()
    assert all(np.array_equal(got[k][0], ref[k][0]) and np.array_equal(got[k][1], ref[k][1]) for k in ref)
    m.shift(tuple(p["origin"]))
    v1, w1 = m.read()
    assert np.array_equal(v0, v1) and np.array_equal(w0, w1)


@settings(max_examples=15, deadline=None)
@given(seed=st.integers(0, 2 ** 31 - 1), reduce=st.sampled_from([0, 1]))
def test_scan_result_independent_of_point_order(seed, reduce):
    """The per-scan volume is an integer reduction: permuting the points of a
    scan changes nothing."""
    p, pts, pose = _room()
    p = dict(p, reduce=reduce)
    perm = np.random.default_rng(seed).permutation(pts.shape[0])
    a, b = oracle.OracleMap(p), oracle.OracleMap(p)
    a.integrate(pts, pose)
    b.integrate(pts[perm], pose)
    va, wa = a.read()
    vb, wb = b.read()
    assert np.array_equal(va, vb) and np.array_equal(wa, wb) and a.stats() == b.stats()
