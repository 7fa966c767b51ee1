"""Checkpoint / resume through tsdf_map_save and tsdf_map_load: the file holds
exactly the oracle's global map (window + store), and a map rebuilt from it
continues bit for bit like the original."""
import numpy as np
import pytest

import oracle
from paper_2310_05766_gb300 import synth
from helpers import run_oracle, workload_steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _words(v, w):
    return v.astype(np.uint16).astype(np.uint32) | (w.astype(np.uint16).astype(np.uint32) << 16)


def _apply(m, steps):
    for st in steps:
        if st[0] == "scan":
            m.integrate(torch.from_numpy(np.ascontiguousarray(st[1], np.float32)).cuda(), st[2])
        else:
            m.shift(st[1])


def _oracle_after(params, steps):
    om = oracle.OracleMap(params)
    for st in steps:
        if st[0] == "scan":
            om.integrate(st[1], st[2])
        else:
            om.shift(st[1])
    return om


def _check_file(path, om):
    from paper_2310_05766_gb300 import binding as b
    params, chunks = b.read_map_file(path)
    ref = om.global_chunks()
    assert tuple(params["origin"]) == om.origin
    assert chunks.keys() == ref.keys()
    for k, (v, w) in ref.items():
        assert np.array_equal(chunks[k], _words(v, w)), k
    return len(ref)


@pytest.mark.parametrize("reduce", [0, 1])
def test_save_load_resume_outdoor(tmp_path, reduce):
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_outdoor(n_scans=14, reduce=reduce)
    steps = workload_steps(w)
    n_shift = sum(1 for st in steps if st[0] == "shift")
    assert n_shift >= 1
    m = b.TsdfMap(w.params)
    path = str(tmp_path / "outdoor.tsdf")
    try:
        _apply(m, steps)
        m.save(path)
        om = _oracle_after(w.params, steps)
        assert om.store_chunks() > 0
        assert _check_file(path, om) > 1000
        m2 = b.TsdfMap.load(path)
        try:
            assert m2.origin == m.origin
            va, wa = m.read()
            vb, wb = m2.read()
            assert np.array_equal(va, vb) and np.array_equal(wa, wb)
            # resume: go back to the first window (its chunks come from the
            # store) and integrate the first scan again, on both maps
            more = [("shift", tuple(w.params["origin"])), ("scan", w.scans[0], w.poses[0])]
            _apply(m, more)
            _apply(m2, more)
            va, wa = m.read()
            vb, wb = m2.read()
            assert np.array_equal(va, vb) and np.array_equal(wa, wb)
            vo, wo, _, _ = run_oracle(w.params, steps + more)
            assert np.array_equal(va, vo) and np.array_equal(wa, wo)
            # the resumed map saves the same global map as the original
            p1, p2 = str(tmp_path / "a.tsdf"), str(tmp_path / "b.tsdf")
            m.save(p1)
            m2.save(p2)
            _, c1 = b.read_map_file(p1)
            _, c2 = b.read_map_file(p2)
            assert c1.keys() == c2.keys() and all(np.array_equal(c1[k], c2[k]) for k in c1)
        finally:
            m2.close()
    finally:
        m.close()


def test_save_empty_and_small_maps(tmp_path):
    from paper_2310_05766_gb300 import binding as b
    p = synth.params_dict((16, 16, 16), 0.1, 0.3, 8, 0.05, 0.05, 3.0, 0, (-8, -8, -8), flags=3)
    m = b.TsdfMap(p)
    path = str(tmp_path / "empty.tsdf")
    try:
        m.save(path)
        params, chunks = b.read_map_file(path)
        assert chunks == {} and params["dims"] == (16, 16, 16) and params["flags"] == 3
        m2 = b.TsdfMap.load(path)
        v, wt = m2.read()
        assert not v.any() and not wt.any()
        m2.close()
        # a random scan with shifts, saved and reloaded at another origin
        rng = np.random.default_rng(5)
        pts = np.zeros((500, 4), np.float32)
        d = rng.normal(size=(500, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pts[:, :3] = d * rng.uniform(0.2, 0.7, (500, 1))
        pose = synth.pose12(synth.rot_zyx(0.4, 0.1, 0.2), np.array([0.02, -0.03, 0.01]))
        steps = [("scan", pts, pose), ("shift", (0, -8, -16)), ("scan", pts, pose), ("shift", (8, 8, 0))]
        _apply(m, steps)
        m.save(path)
        om = _oracle_after(p, steps)
        _check_file(path, om)
        m3 = b.TsdfMap.load(path)
        _apply(m3, [("shift", (-8, -8, -8)), ("scan", pts, pose)])
        v, wt = m3.read()
        vo, wo, _, _ = run_oracle(p, steps + [("shift", (-8, -8, -8)), ("scan", pts, pose)])
        assert np.array_equal(v, vo) and np.array_equal(wt, wo)
        m3.close()
    finally:
        m.close()
