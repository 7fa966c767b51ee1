"""Serving loop: many map sessions, requests arriving in any interleaving,
continuous batching on two streams. Every session's map must be bit-identical
to running its scans alone, in order, through tsdf_integrate / tsdf_shift."""
import numpy as np
import pytest

import oracle
from paper_2310_05766_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MiB = 1 << 20


def _sessions(n, seed):
    out = []
    rng = np.random.default_rng(seed)
    for i in range(n):
        dims = [(128, 128, 64), (256, 256, 64), (128, 128, 128)][i % 3]
        vs = [0.05, 0.064, 0.08, 0.1][int(rng.integers(0, 4))]
        w = synth.workload_outdoor(n_scans=4, seed=500 + seed * 10 + i, reduce=i % 2, beams=[16, 32, 64][i % 3],
                                   azimuths=[512, 1024][i % 2], dims=dims, voxel_size=vs, tau=max(0.2, 2.5 * vs))
        # force a re-centring before the third scan to exercise shifts
        o = w.origins[0]
        w.origins = [o, o, (o[0] + 16, o[1] - 8, o[2]), (o[0] + 16, o[1] - 8, o[2])]
        out.append(w)
    return out


def _alone(b, w):
    m = b.TsdfMap(w.params)
    cur = tuple(w.params["origin"])
    stats = []
    for pts, pose, org in zip(w.scans, w.poses, w.origins):
        if tuple(org) != cur:
            m.shift(org)
            cur = tuple(org)
        m.integrate(torch.from_numpy(pts).cuda(), pose)
        stats.append(m.stats())
    v, wt = m.read()
    m.close()
    return v, wt, stats


def _oracle_session(w):
    """The oracle's map and per-scan counters after a session's scans (and
    shifts) in order."""
    om = oracle.OracleMap(w.params)
    cur = tuple(w.params["origin"])
    stats = []
    for pts, pose, org in zip(w.scans, w.poses, w.origins):
        if tuple(org) != cur:
            om.shift(org)
            cur = tuple(org)
        om.integrate(pts, pose)
        stats.append(om.stats())
    v, wt = om.read()
    om.close()
    return v, wt, stats


@pytest.mark.parametrize("pinned", [False, True])
def test_mixed_equals_alone(pinned):
    """Each session's map is the same in the mix as alone; with pinned
    submissions the server reads the points in place instead of copying."""
    from paper_2310_05766_gb300 import binding as b
    ws = _sessions(6, seed=1)
    held = {}   # pinned submissions must stay alive until their tickets are waited for
    srv = b.tsdf_server_create(hbm_budget_bytes=8 << 30, max_points=1 << 16, max_batch=4, streams=2,
                               max_outstanding=64)
    try:
        sids = [b.tsdf_server_open_session(srv, w.params) for w in ws]
        # interleave: round-robin over sessions, each session's scans in order
        tickets = {i: [] for i in range(len(ws))}
        cur = [tuple(w.params["origin"]) for w in ws]
        order = [(i, k) for k in range(4) for i in np.random.default_rng(3).permutation(len(ws))]
        for i, k in order:
            w = ws[i]
            org = tuple(w.origins[k])
            shift = org if org != cur[i] else None
            cur[i] = org
            pts = w.scans[k]
            if pinned:
                pts = torch.from_numpy(np.ascontiguousarray(pts, np.float32)).pin_memory()
                held[(i, k)] = pts
            tickets[i].append(b.tsdf_server_submit(srv, sids[i], pts, w.poses[k], new_origin=shift))
        results = {i: [b.tsdf_server_wait(srv, t) for t in tickets[i]] for i in tickets}
        st = b.tsdf_server_get_stats(srv)
        assert st["completed"] == 4 * len(ws)
        for i, w in enumerate(ws):
            for r in results[i]:
                assert r["status"] == 0 and r["t_submit_us"] <= r["t_start_us"] <= r["t_done_us"]
            mh = b.tsdf_server_session_map(srv, sids[i])
            o = b.tsdf_get_origin(mh)
            d = w.params["dims"]
            vm, wm = b.tsdf_read(mh, o, tuple(o[a] + d[a] for a in range(3)))
            va, wa, sa = _alone(b, w)
            assert np.array_equal(vm, va) and np.array_equal(wm, wa), f"session {i}"
            assert [r["stats"] for r in results[i]] == sa
        # every session also against the oracle
        for i, w in enumerate(ws):
            vo, wo, so = _oracle_session(w)
            mh = b.tsdf_server_session_map(srv, sids[i])
            o = b.tsdf_get_origin(mh)
            d = w.params["dims"]
            vm, wm = b.tsdf_read(mh, o, tuple(o[a] + d[a] for a in range(3)))
            assert np.array_equal(vm, vo) and np.array_equal(wm, wo), f"session {i} vs oracle"
            assert [r["stats"] for r in results[i]] == so
        assert st["mean_batch"] >= 1.0
    finally:
        b.tsdf_server_destroy(srv)


def test_admission_by_budget_and_back_pressure():
    from paper_2310_05766_gb300 import binding as b
    p = synth.params_dict((256, 256, 128), 0.064, 0.3, 64, 0.006, 0.5, 50.0, 0, (-128, -128, -64))
    # one session: 2^23 voxels * 12 B = 96 MiB + ray buffers + the store's device
    # tier (an eighth of 16384 bricks, rounded up to one 8 MiB segment): 104.2 MiB;
    # a 330 MiB budget admits 3
    srv = b.tsdf_server_create(hbm_budget_bytes=330 * MiB, max_points=1 << 12, max_batch=4, streams=2,
                               max_outstanding=2)
    try:
        sids = [b.tsdf_server_open_session(srv, p) for _ in range(3)]
        with pytest.raises(b.TsdfError) as e:
            b.tsdf_server_open_session(srv, p)
        assert e.value.code == b.TSDF_ERR_ADMISSION
        b.tsdf_server_close_session(srv, sids[0])
        sids[0] = b.tsdf_server_open_session(srv, p)   # admitted once memory is free
        pts = np.zeros((100, 4), np.float32)
        pts[:, 0] = np.linspace(1.0, 5.0, 100)
        pose = synth.pose12(np.eye(3), np.zeros(3))
        t1 = b.tsdf_server_submit(srv, sids[1], pts, pose)
        t2 = b.tsdf_server_submit(srv, sids[1], pts, pose)
        with pytest.raises(b.TsdfError) as e:   # two outstanding: no pinned slab left
            b.tsdf_server_submit(srv, sids[2], pts, pose)
        assert e.value.code == b.TSDF_ERR_BUSY
        with pytest.raises(b.TsdfError) as e:   # requests not yet waited for
            b.tsdf_server_close_session(srv, sids[1])
        assert e.value.code == b.TSDF_ERR_BUSY
        r1 = b.tsdf_server_wait(srv, t1)
        r2 = b.tsdf_server_wait(srv, t2)
        assert r1["stats"]["valid_rays"] == 100 and r2["t_done_us"] >= r1["t_done_us"]
        b.tsdf_server_close_session(srv, sids[1])
        with pytest.raises(b.TsdfError):
            b.tsdf_server_wait(srv, t1)   # each ticket is waited for once
    finally:
        b.tsdf_server_destroy(srv)


def test_submit_many_and_wait_many():
    """Bursts through tsdf_server_submit_many / tsdf_server_wait_many (pinned
    points read in place): every session ends as its scans run alone, and a
    burst larger than the outstanding window is queued up to the window."""
    from paper_2310_05766_gb300 import binding as b
    ws = _sessions(4, seed=9)
    srv = b.tsdf_server_create(hbm_budget_bytes=8 << 30, max_points=1 << 16, max_batch=4, streams=2,
                               max_outstanding=6)
    try:
        sids = [b.tsdf_server_open_session(srv, w.params) for w in ws]
        # scans without window shifts: the first two of each session if they share the origin
        plan = [(i, k) for k in range(2) for i in range(len(ws)) if tuple(ws[i].origins[k]) == tuple(ws[i].params["origin"])]
        pts = [torch.from_numpy(np.ascontiguousarray(ws[i].scans[k], np.float32)).pin_memory() for i, k in plan]
        tickets = b.tsdf_server_submit_many(srv, [sids[i] for i, _ in plan], pts, [ws[i].poses[k] for i, k in plan])
        assert len(tickets) == min(6, len(plan))          # the window holds 6 outstanding requests
        # an unknown ticket in the list is marked, the others are still taken
        res = b.tsdf_server_wait_many(srv, [tickets[0], 1 << 60] + tickets[1:])
        assert res[1]["status"] == b.TSDF_ERR_INVALID and res[1]["ticket"] == 1 << 60
        del res[1]
        assert [r["ticket"] for r in res] == tickets
        rest = b.tsdf_server_submit_many(srv, [sids[i] for i, _ in plan[len(tickets):]], pts[len(tickets):],
                                         [ws[i].poses[k] for i, k in plan[len(tickets):]])
        res += b.tsdf_server_wait_many(srv, rest)
        assert len(res) == len(plan) and all(r["status"] == 0 for r in res)
        for i, w in enumerate(ws):
            ks = [k for j, k in plan if j == i]
            m = b.TsdfMap(w.params)
            for k in ks:
                m.integrate(torch.from_numpy(w.scans[k]).cuda(), w.poses[k])
            va, wa = m.read()
            m.close()
            mh = b.tsdf_server_session_map(srv, sids[i])
            o = b.tsdf_get_origin(mh)
            d = w.params["dims"]
            vm, wm = b.tsdf_read(mh, o, tuple(o[a] + d[a] for a in range(3)))
            assert np.array_equal(vm, va) and np.array_equal(wm, wa)
    finally:
        b.tsdf_server_destroy(srv)


def test_serving_config_shapes_equal_oracle():
    """The serving workload's shapes: 32 sessions (grids 256^3 / 512x512x128,
    voxel 0.05-0.1 m, tau 0.2-0.6 m), two scans each of {16,32,64,128} x
    {1024,2048} points, submitted interleaved over all sessions (batches of up
    to 32 on two streams). Every session's map and counters equal the oracle's."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_2310_05766_gb300 import binding as b
    sess = synth.serving_sessions(32, seed=100)
    rng = synth.SplitMix64(777)
    ws = []
    for sp in sess:
        beams = [16, 32, 64, 128][int(rng.integers(1, 0, 4)[0])]
        az = [1024, 2048][int(rng.integers(1, 0, 2)[0])]
        ws.append(synth.workload_outdoor(n_scans=2, seed=sp["seed"], beams=beams, azimuths=az, dims=sp["dims"],
                                         voxel_size=sp["voxel_size"], tau=sp["tau"]))
    with ThreadPoolExecutor(max_workers=16) as ex:
        ref = list(ex.map(_oracle_session, ws))
    srv = b.tsdf_server_create(hbm_budget_bytes=120 * 10**9, max_points=128 * 2048, max_batch=32, streams=2,
                               max_outstanding=1024)
    try:
        sids = [b.tsdf_server_open_session(srv, w.params) for w in ws]
        order = [(i, k) for k in range(2) for i in np.random.default_rng(5).permutation(len(ws))]
        tickets = {i: [] for i in range(len(ws))}
        # all 64 scans in one call from pinned memory (read in place, so the
        # call queues them at once), so that batches of many sessions form;
        # requests that arrive one at a time are served as they come
        pinned = {(i, k): torch.from_numpy(ws[i].scans[k]).pin_memory() for i, k in order}
        got = b.tsdf_server_submit_many(srv, [sids[i] for i, k in order], [pinned[(i, k)] for i, k in order],
                                        [ws[i].poses[k] for i, k in order])
        assert len(got) == len(order)
        for (i, k), t in zip(order, got):
            tickets[i].append(t)
        for i, w in enumerate(ws):
            res = [b.tsdf_server_wait(srv, t) for t in tickets[i]]
            assert all(r["status"] == 0 for r in res)
            mh = b.tsdf_server_session_map(srv, sids[i])
            o = b.tsdf_get_origin(mh)
            d = w.params["dims"]
            vm, wm = b.tsdf_read(mh, o, tuple(o[a] + d[a] for a in range(3)))
            vo, wo, so = ref[i]
            assert np.array_equal(vm, vo) and np.array_equal(wm, wo), f"session {i}"
            assert [r["stats"] for r in res] == so, f"session {i}"
        assert b.tsdf_server_get_stats(srv)["mean_batch"] > 1.0
    finally:
        b.tsdf_server_destroy(srv)
