"""The seeded input generators (paper_2310_05766_gb300/synth.py), which feed both
the oracle and the CUDA path: the SplitMix64 stream against its published first
outputs, determinism of the workloads, and the sensor model's geometry."""
import math

import numpy as np

from paper_2310_05766_gb300 import synth


def test_splitmix64_published_outputs():
    # first outputs of SplitMix64 (Steele, Lea, Flood 2014) from state 0
    r = synth.SplitMix64(0)
    assert [int(x) for x in r.u64(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # drawing in two calls continues the same stream
    a = synth.SplitMix64(99).u64(10)
    r = synth.SplitMix64(99)
    b = np.concatenate([r.u64(4), r.u64(6)])
    assert np.array_equal(a, b)


def test_uniform_and_normal_ranges():
    r = synth.SplitMix64(5)
    u = r.uniform(100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    z = synth.SplitMix64(6).normal(100000)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
    k = synth.SplitMix64(7).integers(10000, -3, 4)
    assert k.min() == -3 and k.max() == 3


def test_workloads_are_deterministic():
    a, b = synth.workload_room(), synth.workload_room()
    assert np.array_equal(a.scans[0], b.scans[0], equal_nan=True) and np.array_equal(a.poses[0], b.poses[0])
    c, d = synth.workload_outdoor(n_scans=2), synth.workload_outdoor(n_scans=2)
    for s, t in zip(c.scans, d.scans):
        assert np.array_equal(s, t, equal_nan=True)
    assert c.origins == d.origins and c.params == d.params
    e = synth.workload_outdoor(n_scans=1, seed=3)
    assert not np.array_equal(c.scans[0], e.scans[0], equal_nan=True)


def test_beam_directions_and_pose():
    d = synth.beam_directions(4, 8, -15.0, 15.0)
    assert d.shape == (32, 3)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
    # beam-major: the first 8 rows share the lowest elevation, azimuth steps of 45 degrees
    assert np.allclose(d[:8, 2], math.sin(math.radians(-15.0)))
    assert np.allclose(np.arctan2(d[1, 1], d[1, 0]), math.pi / 4)
    R = synth.rot_zyx(0.3, -0.2, 0.1)
    assert np.allclose(R @ R.T, np.eye(3)) and np.isclose(np.linalg.det(R), 1.0)
    p = synth.pose12(R, np.array([1.0, 2.0, 3.0]))
    assert p.dtype == np.float32 and p.shape == (12,)
    assert np.allclose(p.reshape(3, 4)[:, :3], R, atol=1e-7) and np.allclose(p.reshape(3, 4)[:, 3], [1, 2, 3])


def test_outdoor_scan_shape_and_ranges():
    w = synth.workload_outdoor(n_scans=1)
    s = w.scans[0]
    assert s.shape == (128 * 1024, 4) and s.dtype == np.float32
    r = np.linalg.norm(s[:, :3].astype(np.float64), axis=1)
    ok = np.isfinite(r)
    assert ok.mean() > 0.5                       # most beams return
    assert r[ok].max() <= 100.0 + 0.031          # r_max plus the 3-sigma noise bound
    assert np.all(s[ok, 3] == 0.0)
