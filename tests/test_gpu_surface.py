"""Zero-crossing surface points extracted on the GPU (tsdf_extract_surface)
against the oracle's, as exact float sets, on maps built by the GPU path
(which matches the oracle bit for bit) including a ring-wrapped window."""
import numpy as np
import pytest

import oracle
from paper_2310_05766_gb300 import synth
from helpers import workload_steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sorted(p):
    p = np.asarray(p, np.float32)
    return p[np.lexsort((p[:, 3], p[:, 2], p[:, 1], p[:, 0]))]


def _build(params, steps):
    from paper_2310_05766_gb300 import binding as b
    m = b.TsdfMap(params)
    om = oracle.OracleMap(params)
    for st in steps:
        if st[0] == "scan":
            m.integrate(torch.from_numpy(np.ascontiguousarray(st[1], np.float32)).cuda(), st[2])
            om.integrate(st[1], st[2])
        else:
            m.shift(st[1])
            om.shift(st[1])
    return m, om


@pytest.mark.parametrize("min_weight", [1, 2])
def test_surface_room_exact(min_weight):
    w = synth.workload_room()
    m, om = _build(w.params, workload_steps(w) + [("scan", w.scans[0], w.poses[0])])
    try:
        got = m.surface(min_weight).cpu().numpy()
        ref = om.surface(min_weight)
        assert len(ref) > 10000
        assert np.array_equal(_sorted(got), _sorted(ref))
    finally:
        m.close()


def test_surface_outdoor_after_shift_exact():
    w = synth.workload_outdoor(n_scans=12)
    steps = workload_steps(w)
    assert any(st[0] == "shift" for st in steps)
    m, om = _build(w.params, steps)
    try:
        got = m.surface().cpu().numpy()
        ref = om.surface()
        assert len(ref) > 100000
        assert np.array_equal(_sorted(got), _sorted(ref))
    finally:
        m.close()


def test_surface_capacity_and_arguments():
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_room()
    m, om = _build(w.params, workload_steps(w))
    try:
        n_ref = len(om.surface())
        small = torch.zeros((100, 4), dtype=torch.float32, device="cuda")
        pts, n = b.tsdf_extract_surface(m.handle, 1, small)
        assert n == n_ref and pts.shape[0] == 100
        full = _sorted(om.surface())
        got = pts.cpu().numpy()
        # every written point is one of the oracle's
        idx = np.searchsorted(full[:, 0], got[:, 0])
        assert np.all(idx < len(full))
        for opt in [0, 40000]:
            with pytest.raises(b.TsdfError):
                b.tsdf_extract_surface(m.handle, opt, small)
    finally:
        m.close()


def _canon_tris(t):
    """Triangles as sorted rows, each rotated so its smallest vertex comes first
    (keeps the orientation)."""
    t = np.asarray(t, np.float32).reshape(-1, 3, 3)
    out = []
    for tri in t:
        k = min(range(3), key=lambda i: tuple(tri[i]))
        r = np.roll(tri, -k, axis=0)
        out.append(r.reshape(9))
    out = np.array(out, np.float32).reshape(-1, 9)
    return out[np.lexsort(out.T[::-1])]


@pytest.mark.parametrize("min_weight", [1, 3])
def test_mesh_room_exact(min_weight):
    w = synth.workload_room()
    m, om = _build(w.params, workload_steps(w) + [("scan", w.scans[0], w.poses[0])])
    try:
        got = m.mesh(min_weight).cpu().numpy()
        ref = om.mesh(min_weight)
        assert len(ref) > (5000 if min_weight == 1 else 1000)
        assert np.array_equal(_canon_tris(got), _canon_tris(ref))
    finally:
        m.close()


def test_mesh_outdoor_after_shift_exact():
    w = synth.workload_outdoor(n_scans=12)
    m, om = _build(w.params, workload_steps(w))
    try:
        got = m.mesh().cpu().numpy()
        ref = om.mesh()
        assert len(ref) > 100000
        assert np.array_equal(_canon_tris(got), _canon_tris(ref))
    finally:
        m.close()
