"""The global chunk store behind the ring-buffered window (the paper's
Introduction: the local map is shifted, map parts that leave it are written
out and previously mapped parts are read back). Only chunks that hold data are
stored; the store's device tier is bounded and spills its oldest chunks to
pinned host memory, which the shift kernel reads and writes in place. Every
window is compared with the oracle, whose store keeps exactly the non-empty
chunks (std::map, no tiers)."""
import os

import numpy as np
import pytest

import oracle
from paper_2310_05766_gb300 import synth
from helpers import assert_same, run_gpu, run_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MiB = 1 << 20


def _ball_scan(seed=21, n=3000):
    rng = np.random.default_rng(seed)
    pts = np.zeros((n, 4), np.float32)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts[:, :3] = d * rng.uniform(0.5, 2.8, (n, 1))
    return pts


def test_walk_over_empty_ground_keeps_device_bytes_flat():
    """A 64^3 window with data in one corner walks 40 window widths away over
    empty ground and back. Empty leaving chunks are dropped, so after the first
    shift the map's device memory stays the same; the corner comes back intact."""
    from paper_2310_05766_gb300 import binding as b
    p = synth.params_dict((64, 64, 64), 0.1, 0.3, 64, 0.05, 0.3, 3.0, 0, (0, 0, 0))
    rng = np.random.default_rng(3)
    v0 = np.zeros((64, 64, 64), np.int16)
    w0 = np.zeros((64, 64, 64), np.int16)
    w0[:24, :20, :16] = rng.integers(1, 64, (24, 20, 16))
    v0[:24, :20, :16] = rng.integers(-32767, 32768, (24, 20, 16))
    m = b.TsdfMap(p)
    om = oracle.OracleMap(p)
    try:
        m.write(v0, w0)
        om.load_window(v0, w0)
        sizes = []
        xs = list(range(1, 41)) + list(range(39, -1, -1))
        for k, xi in enumerate(xs):
            o = (64 * xi, 0, 0)
            m.shift(o)
            om.shift(o)
            sizes.append(b.tsdf_map_device_bytes(m.handle))
        st = b.tsdf_get_store_stats(m.handle)
        assert len(set(sizes)) == 1, sizes[:5]
        assert st["device_chunks"] == 0 and st["host_chunks"] == 0   # the corner is back in the window
        assert st["dropped"] >= 78 * 512 - 3 * 3 * 2
        vg, wg = m.read()
        vo, wo = om.read()
        assert np.array_equal(vg, vo) and np.array_equal(wg, wo)
        assert np.array_equal(vg, v0) and np.array_equal(wg, w0)
    finally:
        m.close()
        om.close()


@pytest.mark.parametrize("age", [0, 3])
def test_store_spills_to_host_memory_and_reads_back(age):
    """The 64^3 window moved by its own size 26 times with a scan at every
    position and back, with the device tier limited to one 8 MiB segment (4096
    chunks, fewer than the walk stores) and, with age 3, chunks stored three
    shifts ago moved to host memory. Compared with the oracle at three points of
    the walk back, whose chunks come from the host tier; device memory bounded."""
    from paper_2310_05766_gb300 import binding as b
    p = synth.params_dict((64, 64, 64), 0.1, 0.3, 64, 0.05, 0.3, 3.0, 0, (0, 0, 0))
    pts = _ball_scan()
    steps = []
    checks = []
    xs = list(range(0, 27)) + list(range(25, -1, -1))
    for k, xi in enumerate(xs):
        origin = (64 * xi, 0, 0)
        if k > 0:
            steps.append(("shift", origin))
        t = np.array([(origin[0] + 32) * 0.1, 3.2, 3.2])
        steps.append(("scan", pts, synth.pose12(synth.rot_zyx(0.1 * k, 0.0, 0.0), t)))
        if k > 26 and xi in (24, 12, 0):
            checks.append((xi, len(steps)))
    opts = {b.TSDF_OPT_STORE_DEVICE_CHUNKS: 4096, b.TSDF_OPT_STORE_SPILL_AGE: age}
    for xi, n in checks:
        g = run_gpu(p, steps[:n], torch, options=opts)
        o = run_oracle(p, steps[:n])
        assert_same(g, o, f"spilled store, back at x = {64 * xi}")
    # the store's tiers over the whole walk out
    m = b.TsdfMap(p)
    try:
        for opt, val in opts.items():
            b.tsdf_set_option(m.handle, opt, val)
        first = None
        for st in steps[:53]:
            if st[0] == "scan":
                m.integrate(torch.from_numpy(st[1]).cuda(), st[2])
            else:
                m.shift(st[1])
                if first is None:
                    first = b.tsdf_map_device_bytes(m.handle)
        ss = b.tsdf_get_store_stats(m.handle)
        assert ss["device_capacity"] == 4096 and ss["device_chunks"] <= 4096
        assert ss["host_chunks"] > 0 and ss["spilled"] > 0
        assert b.tsdf_map_device_bytes(m.handle) == first
        om = oracle.OracleMap(p)
        for st in steps[:53]:
            if st[0] == "scan":
                om.integrate(st[1], st[2])
            else:
                om.shift(st[1])
        o = om.origin
        lo = [o[a] // 8 for a in range(3)]
        outside = [k for k in om.global_chunks() if any(not (lo[a] <= k[a] < lo[a] + 8) for a in range(3))]
        assert ss["device_chunks"] + ss["host_chunks"] == len(outside)
        om.close()
    finally:
        m.close()


def test_saved_map_includes_host_tier_chunks(tmp_path):
    """A map whose store spilled to host memory saves every stored chunk: the
    file holds exactly the oracle's global map, and the reloaded map continues
    like the original and the oracle."""
    from paper_2310_05766_gb300 import binding as b
    p = synth.params_dict((64, 64, 64), 0.1, 0.3, 64, 0.05, 0.3, 3.0, 0, (0, 0, 0))
    pts = _ball_scan(seed=5)
    m = b.TsdfMap(p)
    om = oracle.OracleMap(p)
    m2 = None
    try:
        b.tsdf_set_option(m.handle, b.TSDF_OPT_STORE_DEVICE_CHUNKS, 4096)
        b.tsdf_set_option(m.handle, b.TSDF_OPT_STORE_SPILL_AGE, 1)
        for k in range(12):
            o = (64 * k, 0, 0)
            if k:
                m.shift(o)
                om.shift(o)
            pose = synth.pose12(synth.rot_zyx(0.2 * k, 0.0, 0.0), np.array([(o[0] + 32) * 0.1, 3.2, 3.2]))
            m.integrate(torch.from_numpy(pts).cuda(), pose)
            om.integrate(pts, pose)
        assert b.tsdf_get_store_stats(m.handle)["host_chunks"] > 0
        path = str(tmp_path / "map.tsdf")
        m.save(path)
        _, chunks = b.read_map_file(path)
        ref = om.global_chunks()
        assert chunks.keys() == ref.keys()
        for key, (v, w) in ref.items():
            words = v.astype(np.uint16).astype(np.uint32) | (w.astype(np.uint16).astype(np.uint32) << 16)
            assert np.array_equal(chunks[key], words), key
        m2 = b.TsdfMap.load(path)
        for mm in (m, m2):
            mm.shift((0, 0, 0))
        om.shift((0, 0, 0))
        vo, wo = om.read()
        for mm in (m, m2):
            vg, wg = mm.read()
            assert np.array_equal(vg, vo) and np.array_equal(wg, wo)
    finally:
        m.close()
        om.close()
        if m2 is not None:
            m2.close()


def test_store_file_tier_reads_back_exactly(tmp_path):
    """The walk of the host-tier test with a third tier in a file: the device
    tier limited to one segment (4096 chunks), the host tier kept to 256
    chunks at the start of every shift, older chunks written to a scratch file
    by the map's writer thread. The map saved at the far end holds exactly the
    oracle's global map (file-tier chunks included); on the way back the
    window equals the oracle's at every position (chunks read back from the
    file, or from the write queue); the scratch file goes with the map."""
    from paper_2310_05766_gb300 import binding as b
    p = synth.params_dict((64, 64, 64), 0.1, 0.3, 64, 0.05, 0.3, 3.0, 0, (0, 0, 0))
    pts = torch.from_numpy(_ball_scan(seed=33)).cuda()
    pts_np = pts.cpu().numpy()
    scratch = str(tmp_path / "store.bin")
    m = b.TsdfMap(p)
    om = oracle.OracleMap(p)
    try:
        b.tsdf_set_option(m.handle, b.TSDF_OPT_STORE_DEVICE_CHUNKS, 4096)
        m.set_store_file(scratch, 256)
        with pytest.raises(b.TsdfError):
            b.tsdf_map_set_store_file(m.handle, scratch, 256)   # once per map
        assert os.path.exists(scratch)
        xs = list(range(0, 27)) + list(range(25, -1, -1))
        checked = 0
        for k, xi in enumerate(xs):
            o = (64 * xi, 0, 0)
            if k:
                m.shift(o)
                om.shift(o)
            pose = synth.pose12(synth.rot_zyx(0.1 * k, 0.0, 0.0), np.array([(o[0] + 32) * 0.1, 3.2, 3.2]))
            m.integrate(pts, pose)
            om.integrate(pts_np, pose)
            if k == 26:
                st = b.tsdf_get_store_stats(m.handle)
                assert st["to_file"] > 0 and st["file_chunks"] > 0
                path = str(tmp_path / "map.tsdf")
                m.save(path)
                _, chunks = b.read_map_file(path)
                ref = om.global_chunks()
                assert chunks.keys() == ref.keys()
                for key, (v, w) in ref.items():
                    words = v.astype(np.uint16).astype(np.uint32) | (w.astype(np.uint16).astype(np.uint32) << 16)
                    assert np.array_equal(chunks[key], words), key
            if k > 26:
                vg, wg = m.read()
                vo, wo = om.read()
                assert np.array_equal(vg, vo) and np.array_equal(wg, wo), f"back at x = {64 * xi}"
                checked += 1
        st = m.store_stats()
        assert checked == 26 and st["from_file"] > 0
        assert st["device_capacity"] == 4096
        o = om.origin
        lo = [o[a] // 8 for a in range(3)]
        outside = [q for q in om.global_chunks() if any(not (lo[a] <= q[a] < lo[a] + 8) for a in range(3))]
        assert st["device_chunks"] + st["host_chunks"] + st["file_chunks"] == len(outside)
    finally:
        m.close()
        om.close()
    assert not os.path.exists(scratch)


def test_serving_charges_the_store_reservation():
    """Each session's store device tier is reserved and charged when it opens:
    a budget that fits two sessions with their reservations refuses the third
    (it would fit without them). A session that shifts through more chunks
    than its reservation spills to host memory, allocates no device memory,
    and equals the oracle."""
    from paper_2310_05766_gb300 import binding as b
    p = synth.params_dict((64, 64, 64), 0.1, 0.3, 64, 0.05, 0.3, 3.0, 0, (0, 0, 0))
    # per session: 2^18 voxels * 12 B + 512 bricks * 5 + 4096 points * 32 + 8192
    # = 3.02 MiB, plus the store reservation: 4096 chunks * 2 KiB = 8 MiB
    srv = b.tsdf_server_create(hbm_budget_bytes=24 * MiB, max_points=1 << 12, max_batch=4, streams=2,
                               max_outstanding=64, store_chunks=4096)
    try:
        s1 = b.tsdf_server_open_session(srv, p)
        s2 = b.tsdf_server_open_session(srv, p)
        with pytest.raises(b.TsdfError) as e:
            b.tsdf_server_open_session(srv, p)
        assert e.value.code == b.TSDF_ERR_ADMISSION
        assert b.tsdf_server_get_stats(srv)["used_bytes"] > 2 * 11 * MiB
        mh = b.tsdf_server_session_map(srv, s1)
        before = b.tsdf_map_device_bytes(mh)
        pts = _ball_scan(seed=9, n=3000)[:4096]
        om = oracle.OracleMap(p)
        tickets = []
        for k in range(30):
            o = (64 * k, 0, 0)
            pose = synth.pose12(synth.rot_zyx(0.3 * k, 0.0, 0.0), np.array([(o[0] + 32) * 0.1, 3.2, 3.2]))
            tickets.append(b.tsdf_server_submit(srv, s1, pts, pose, new_origin=o if k else None))
            if k:
                om.shift(o)
            om.integrate(pts, pose)
        for t in tickets:
            assert b.tsdf_server_wait(srv, t)["status"] == 0
        st = b.tsdf_get_store_stats(mh)
        assert st["host_chunks"] > 0 and st["device_capacity"] == 4096
        assert b.tsdf_map_device_bytes(mh) == before
        o = b.tsdf_get_origin(mh)
        vm, wm = b.tsdf_read(mh, o, (o[0] + 64, o[1] + 64, o[2] + 64))
        vo, wo = om.read()
        assert np.array_equal(vm, vo) and np.array_equal(wm, wo)
        om.close()
        b.tsdf_server_close_session(srv, s2)
    finally:
        b.tsdf_server_destroy(srv)


def test_one_km_drive_bounded_device_memory_exact_at_every_reentry():
    """A 1 km drive (500 m out along x and back, a scan every 4 m) with a 32 x 32
    x 8 m window (128 x 128 x 32 at 0.25 m) over a seeded ground-and-boxes
    scene, the store's device tier limited to one segment (4096 chunks, fewer
    than the drive stores): device memory stays bounded, chunks spill to host
    memory, and on the way back the window equals the oracle's at every
    position (every re-entered chunk read back exactly)."""
    from paper_2310_05766_gb300 import binding as b
    vs, dims = 0.25, (128, 128, 32)
    xs = [4.0 * i for i in range(126)] + [4.0 * i for i in range(124, -1, -1)]
    path = np.array([[x, 0.0] for x in xs[:126]])
    scene = synth.outdoor_scene(41, path, n_boxes=400, n_cyl=100, extent=520.0)
    dirs = synth.beam_directions(16, 360, -15.0, 15.0)
    rng = synth.SplitMix64(42)
    p = synth.params_dict(dims, vs, 0.75, 64, synth.delta_z_for(30.0, 16), 0.5, 40.0, 0,
                          synth.window_origin((0.0, 0.0, 0.0), dims, vs))
    m = b.TsdfMap(p)
    om = oracle.OracleMap(p)
    try:
        b.tsdf_set_option(m.handle, b.TSDF_OPT_STORE_DEVICE_CHUNKS, 4096)
        sizes = []
        checked = 0
        for k, x in enumerate(xs):
            R = synth.rot_zyx(0.05 * np.sin(0.1 * k))
            t = np.array([x, 0.0, 0.0])
            o = synth.window_origin(t, dims, vs)
            if k:
                m.shift(o)
                om.shift(o)
                sizes.append(b.tsdf_map_device_bytes(m.handle))
            pts = synth.make_scan(scene, R, t, dirs, 0.01, rng, r_max=40.0)
            pose = synth.pose12(R, t)
            m.integrate(torch.from_numpy(pts).cuda(), pose)
            om.integrate(pts, pose)
            if k > 125:   # on the way back: every position
                vg, wg = m.read()
                vo, wo = om.read()
                assert np.array_equal(vg, vo) and np.array_equal(wg, wo), f"position {k} (x = {x})"
                checked += 1
        st = b.tsdf_get_store_stats(m.handle)
        assert checked == 125
        assert st["spilled"] > 0 and st["device_capacity"] == 4096
        assert max(sizes) == sizes[0]          # bounded: the device tier never grew past its first segment
        # the store holds exactly the oracle's non-empty chunks outside the window
        # (the oracle's own store also keeps copies of chunks that re-entered)
        o = om.origin
        lo = [o[a] // 8 for a in range(3)]
        outside = [k for k in om.global_chunks() if any(not (lo[a] <= k[a] < lo[a] + dims[a] // 8) for a in range(3))]
        assert len(outside) == st["device_chunks"] + st["host_chunks"]
    finally:
        m.close()
        om.close()
