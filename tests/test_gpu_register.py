"""Scan-to-map registration on the GPU (tsdf_register_system / tsdf_register)
against the oracle: the normal equations agree to binary64 summation order
(the per-point arithmetic is the same), Gauss-Newton follows the same path,
and an exact box field gives back a perturbed pose."""
import numpy as np
import pytest

import oracle
from paper_2310_05766_gb300 import synth
from helpers import workload_steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _box_field(vs=0.05, tau=0.2, half=(0.6, 0.4, 0.3), rot=(0.3, 0.2, 0.1)):
    p = synth.params_dict((64, 64, 64), vs, tau, 64, 0.0, 0.1, 10.0, 0, (-32, -32, -32))
    Rb = synth.rot_zyx(*rot)
    half = np.array(half)
    g = np.stack(np.meshgrid(np.arange(-32, 32), np.arange(-32, 32), np.arange(-32, 32), indexing="ij"), -1)
    cen = (g[..., ::-1] + 0.5) * vs
    qd = np.abs(cen @ Rb) - half
    sdf = np.linalg.norm(np.maximum(qd, 0), axis=-1) + np.minimum(qd.max(-1), 0)
    v = np.rint(np.clip(sdf, -tau, tau) * 32767 / tau).astype(np.int16)
    rng = np.random.default_rng(0)
    n = 4000
    face = rng.integers(0, 6, n)
    u = rng.uniform(-1, 1, (n, 3)) * half
    ax = face % 3
    u[np.arange(n), ax] = np.where(face < 3, 1.0, -1.0) * half[ax]
    pts = np.zeros((n, 4), np.float32)
    pts[:, :3] = u @ Rb.T
    return p, v, np.ones_like(v), pts


def _same_system(a, b):
    assert a[28] == b[28]
    scale = np.abs(b).max()
    assert np.allclose(a, b, rtol=1e-9, atol=1e-12 * scale), np.max(np.abs(a - b))


def test_register_box_field_system_and_recovery():
    from paper_2310_05766_gb300 import binding as b
    p, v, w, pts = _box_field()
    m = b.TsdfMap(p)
    om = oracle.OracleMap(p)
    om.load_window(v, w)
    try:
        m.write(v, w)
        pd = torch.from_numpy(pts).cuda()
        for pose in [synth.pose12(np.eye(3), np.zeros(3)),
                     synth.pose12(synth.rot_zyx(0.02, -0.01, 0.015), np.array([0.02, -0.03, 0.01]))]:
            _same_system(b.tsdf_register_system(m.handle, pd, pose), om.register_system(pts, pose))
        start = synth.pose12(synth.rot_zyx(np.deg2rad(1.0), np.deg2rad(-0.7), np.deg2rad(0.5)),
                             np.array([0.03, -0.02, 0.025]))
        got, res = b.tsdf_register(m.handle, pd, start, iterations=6)
        ref = start
        for _ in range(res["iterations"]):
            ref, _ = oracle.pose_update(ref, om.register_system(pts, ref))
        assert np.allclose(got, ref, atol=2e-6)
        P = got.reshape(3, 4).astype(np.float64)
        ang = np.rad2deg(np.arccos(np.clip((np.trace(P[:, :3]) - 1) / 2, -1, 1)))
        assert np.linalg.norm(P[:, 3]) < 5e-4 and ang < 0.1
        assert res["used_points"] == 4000
    finally:
        m.close()


def test_register_outdoor_scan_against_its_map():
    """Maps built by integrating six outdoor scans (identical on both sides);
    the seventh scan from a perturbed pose: same normal equations, same
    Gauss-Newton iterates, and the error shrinks."""
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_outdoor(n_scans=8)
    steps = workload_steps(w, 6)
    assert all(st[0] == "scan" for st in steps)
    m = b.TsdfMap(w.params)
    om = oracle.OracleMap(w.params)
    try:
        for st in steps:
            m.integrate(torch.from_numpy(st[1]).cuda(), st[2])
            om.integrate(st[1], st[2])
        true = w.poses[6].reshape(3, 4).astype(np.float64)
        Rp = synth.rot_zyx(np.deg2rad(0.8), np.deg2rad(0.3), np.deg2rad(-0.3))
        start = np.concatenate([Rp @ true[:, :3], (true[:, 3] + np.array([0.04, -0.03, 0.02]))[:, None]],
                               axis=1).astype(np.float32).reshape(12)
        pts = w.scans[6]
        pd = torch.from_numpy(pts).cuda()
        s_gpu = b.tsdf_register_system(m.handle, pd, start)
        s_orc = om.register_system(pts, start)
        assert s_orc[28] > 50000
        _same_system(s_gpu, s_orc)
        got, res = b.tsdf_register(m.handle, pd, start, iterations=4)
        ref = start
        for _ in range(res["iterations"]):
            ref, _ = oracle.pose_update(ref, om.register_system(pts, ref))
        assert np.allclose(got, ref, atol=1e-5)
        # the rotation error and the residual shrink (translation converges
        # slowly on this projective, plane-dominated field)
        def ang(P):
            dR = P.reshape(3, 4)[:, :3].astype(np.float64) @ true[:, :3].T
            return np.rad2deg(np.arccos(np.clip((np.trace(dR) - 1) / 2, -1, 1)))
        assert ang(got) < 0.7 * ang(start)
        assert res["rms"] < np.sqrt(s_orc[27] / s_orc[28])
    finally:
        m.close()


def test_register_degenerate_and_bad_arguments():
    from paper_2310_05766_gb300 import binding as b
    p, v, w, pts = _box_field()
    m = b.TsdfMap(p)
    try:
        pose = synth.pose12(np.eye(3), np.zeros(3))
        far = torch.full((100, 4), 50.0, dtype=torch.float32, device="cuda")   # outside the window
        with pytest.raises(b.TsdfError) as ei:
            b.tsdf_register(m.handle, far, pose, iterations=3)
        assert ei.value.code == b.TSDF_ERR_DEGENERATE
        assert np.all(b.tsdf_register_system(m.handle, far, pose) == 0)
        pd = torch.from_numpy(pts).cuda()
        with pytest.raises(b.TsdfError):
            b.tsdf_register(m.handle, pd, pose, iterations=0)
        with pytest.raises(b.TsdfError):
            b.tsdf_register_system(m.handle, pd, pose, min_weight=0)
    finally:
        m.close()
