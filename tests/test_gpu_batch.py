"""Batched integration (one persistent cooperative launch for many maps) against
the per-map path and the oracle: every map's grid and counters bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2310_05766_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class _DevView:
    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<u4", "data": (ptr, False), "version": 2}


def _grid(b, m):
    d = m.params["dims"]
    return torch.as_tensor(_DevView(b.tsdf_grid_device_ptr(m.handle), d[0] * d[1] * d[2]), device="cuda")


def _small_batch(n_maps, seed, reduce_mix=True):
    ws = synth.workload_batch(n_maps=n_maps, seed=seed, dims_choices=[(128, 128, 64), (256, 256, 64), (64, 64, 64)])
    if reduce_mix:
        for i, w in enumerate(ws):
            w.params["reduce"] = i % 2
    return ws


def _run_batch(b, ws, batch=None, prefill_steps=0, options=None):
    maps = [b.TsdfMap(w.params) for w in ws]
    pts = [torch.from_numpy(w.scans[0]).cuda() for w in ws]
    poses = [w.poses[0] for w in ws]
    own = batch is None
    if own:
        batch = b.tsdf_batch_create(len(ws))
    for opt, val in (options or {}).items():
        b.tsdf_batch_set_option(batch, opt, val)
    for _ in range(1 + prefill_steps):
        b.tsdf_batch_integrate(batch, maps, pts, poses)
    assert b.tsdf_batch_sync(batch) == b.TSDF_OK
    if own:
        b.tsdf_batch_destroy(batch)
    return maps


def _run_single(b, ws, repeats=1):
    maps = [b.TsdfMap(w.params) for w in ws]
    for _ in range(repeats):
        for m, w in zip(maps, ws):
            m.integrate(torch.from_numpy(w.scans[0]).cuda(), w.poses[0])
    torch.cuda.synchronize()
    return maps


def _same(b, ma, mb):
    for x, y in zip(ma, mb):
        assert torch.equal(_grid(b, x), _grid(b, y))
        assert x.stats() == y.stats()


def test_batch_matches_oracle_and_single():
    from paper_2310_05766_gb300 import binding as b
    ws = _small_batch(6, seed=5)
    mb = _run_batch(b, ws)
    ms = _run_single(b, ws)
    _same(b, mb, ms)
    for m, w in zip(mb[:3], ws[:3]):
        om = oracle.OracleMap(w.params)
        om.integrate(w.scans[0], w.poses[0])
        vo, wo = om.read()
        vg, wg = m.read()
        assert np.array_equal(vg, vo) and np.array_equal(wg, wo)
        assert m.stats() == om.stats()
    for m in mb + ms:
        m.close()


@pytest.mark.parametrize("config", range(13))
@pytest.mark.parametrize("graph,cta_cache", [(0, 1), (1, 1), (1, 0)])
def test_batch_every_config_same_result(config, graph, cta_cache):
    from paper_2310_05766_gb300 import binding as b
    ws = _small_batch(5, seed=11)
    mb = _run_batch(b, ws, prefill_steps=1,
                    options={b.TSDF_BATCH_OPT_CONFIG: config, b.TSDF_BATCH_OPT_GRAPH: graph,
                             b.TSDF_BATCH_OPT_CTA_BRICK_CACHE: cta_cache})
    ms = _run_single(b, ws, repeats=2)
    _same(b, mb, ms)
    for m in mb + ms:
        m.close()


@pytest.mark.parametrize("cta_cache", [1, 0])
def test_batch_of_identical_maps(cta_cache):
    """Eight maps with the same parameters and the same scan in one batch:
    the warps of a CTA mark equal brick numbers of different maps, which the
    shared brick cache must keep apart (its keys carry the map). Every map
    equals the per-map call."""
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_outdoor(n_scans=1)
    ws = [w] * 8
    for config in (0, 8, 9):
        mb = _run_batch(b, ws, options={b.TSDF_BATCH_OPT_CONFIG: config, b.TSDF_BATCH_OPT_CTA_BRICK_CACHE: cta_cache})
        ms = _run_single(b, ws[:1])
        for m in mb:
            assert torch.equal(_grid(b, m), _grid(b, ms[0]))
            assert m.stats() == ms[0].stats()
        for m in mb + ms:
            m.close()


def test_batch_autotune_settles_and_is_exact():
    from paper_2310_05766_gb300 import binding as b
    ws = _small_batch(4, seed=13)
    batch = b.tsdf_batch_create(8)
    mb = _run_batch(b, ws, batch=batch, prefill_steps=29)   # 13 configurations timed twice each
    cfg = b.tsdf_batch_get_config(batch)
    b.tsdf_batch_integrate(batch, mb, [torch.from_numpy(w.scans[0]).cuda() for w in ws], [w.poses[0] for w in ws])
    assert b.tsdf_batch_sync(batch) == b.TSDF_OK
    cfg = b.tsdf_batch_get_config(batch)
    assert cfg["tuned"], cfg
    assert cfg["threads_per_cta"] in (128, 256, 512) and cfg["ctas"] >= 1 and cfg["apply_voxel_pairs"] in (2, 8)
    ms = _run_single(b, ws, repeats=31)
    _same(b, mb, ms)
    b.tsdf_batch_destroy(batch)
    for m in mb + ms:
        m.close()


def test_batch_sort_overflow_matches_single():
    """Sort configuration with a pair capacity far below the scans' samples
    (the overflow path) in one batched launch: equal to the per-map path."""
    from paper_2310_05766_gb300 import binding as b
    ws = _small_batch(4, seed=23)
    maps = [b.TsdfMap(w.params) for w in ws]
    for m in maps:
        b.tsdf_set_option(m.handle, b.TSDF_OPT_SORT_CAPACITY, 4096)
    batch = b.tsdf_batch_create(8)
    b.tsdf_batch_set_option(batch, b.TSDF_BATCH_OPT_CONFIG, 6)
    pts = [torch.from_numpy(w.scans[0]).cuda() for w in ws]
    for _ in range(2):
        b.tsdf_batch_integrate(batch, maps, pts, [w.poses[0] for w in ws])
    assert b.tsdf_batch_sync(batch) == b.TSDF_OK
    assert b.tsdf_batch_get_config(batch)["reduction"] == b.TSDF_REDUCTION_SORT
    b.tsdf_batch_destroy(batch)
    ms = _run_single(b, ws, repeats=2)
    _same(b, maps, ms)
    for m in maps + ms:
        m.close()


def test_batch_flags_match_single():
    """Maps with different reading flags in one batched launch: each equals
    its own per-map integration (and so the oracle, which the per-map path
    matches)."""
    from paper_2310_05766_gb300 import binding as b
    ws = _small_batch(6, seed=19)
    for i, w in enumerate(ws):
        w.params["flags"] = i % 4
    mb = _run_batch(b, ws, prefill_steps=1)
    ms = _run_single(b, ws, repeats=2)
    _same(b, mb, ms)
    for m, w in zip(mb[1:4], ws[1:4]):
        om = oracle.OracleMap(w.params)
        om.integrate(w.scans[0], w.poses[0])
        om.integrate(w.scans[0], w.poses[0])
        vo, wo = om.read()
        vg, wg = m.read()
        assert np.array_equal(vg, vo) and np.array_equal(wg, wo)
    for m in mb + ms:
        m.close()


def test_batch_uneven_sizes_and_empty_scans():
    from paper_2310_05766_gb300 import binding as b
    ws = _small_batch(5, seed=17)
    ws[1].scans[0] = ws[1].scans[0][:0]           # empty scan
    ws[3].scans[0] = ws[3].scans[0][:37]          # ragged tail
    mb = _run_batch(b, ws)
    ms = _run_single(b, ws)
    _same(b, mb, ms)
    assert mb[1].stats() == dict(valid_rays=0, hits=0, touched=0)
    for m in mb + ms:
        m.close()


def _oracle_maps(ws, threads=16):
    """The oracle's map of every workload (one scan each), computed on host
    threads (each map is independent; the oracle calls release the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(w):
        om = oracle.OracleMap(w.params)
        om.integrate(w.scans[0], w.poses[0])
        return om

    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, ws))


def test_batched_64_maps_full_size():
    """64 maps, beams {16..128} x azimuths {512..2048}, grids 256^3 / 512x512x128 at
    0.064 m: one batched launch equals 64 per-map calls, and every one of the 64
    maps equals the oracle (whole window, values and weights, and counters)."""
    from paper_2310_05766_gb300 import binding as b
    ws = synth.workload_batch(n_maps=64, seed=3)
    mb = _run_batch(b, ws)
    ms = _run_single(b, ws)
    _same(b, mb, ms)
    for m in ms:
        m.close()
    oms = _oracle_maps(ws)
    for k, om in enumerate(oms):
        assert mb[k].stats() == om.stats(), k
        vo, wo = om.read()
        vg, wg = mb[k].read()
        assert np.array_equal(vg, vo) and np.array_equal(wg, wo), k
        om.close()
        mb[k].close()


def test_batched_64_maps_every_configuration():
    """The 64-map batch under every tuning configuration, launch shapes
    included (CTAs of 128, 256 and 512 threads, 2 CTAs per SM, quarter-brick
    apply tasks): each equal to the 64 per-map calls."""
    from paper_2310_05766_gb300 import binding as b
    ws = synth.workload_batch(n_maps=64, seed=3)
    ms = _run_single(b, ws)
    shapes = set()
    for config in range(13):
        batch = b.tsdf_batch_create(64)
        mb = _run_batch(b, ws, batch=batch, options={b.TSDF_BATCH_OPT_CONFIG: config})
        c = b.tsdf_batch_get_config(batch)
        shapes.add((c["threads_per_cta"], c["apply_voxel_pairs"], c["ctas"]))
        b.tsdf_batch_destroy(batch)
        _same(b, mb, ms)
        for m in mb:
            m.close()
    assert len(shapes) >= 4
    for m in ms:
        m.close()


def test_batch_rejects_bad_arguments():
    from paper_2310_05766_gb300 import binding as b
    ws = _small_batch(2, seed=19)
    maps = [b.TsdfMap(w.params) for w in ws]
    pts = [torch.from_numpy(w.scans[0]).cuda() for w in ws]
    batch = b.tsdf_batch_create(2)
    try:
        with pytest.raises(b.TsdfError):   # the same map twice
            b.tsdf_batch_integrate(batch, [maps[0], maps[0]], pts, [ws[0].poses[0]] * 2)
        with pytest.raises(b.TsdfError):   # more maps than the object holds
            b.tsdf_batch_integrate(batch, maps + maps[:1], pts + pts[:1], [w.poses[0] for w in ws] + [ws[0].poses[0]])
        with pytest.raises(b.TsdfError):
            b.tsdf_batch_set_option(batch, b.TSDF_BATCH_OPT_CONFIG, 13)
    finally:
        b.tsdf_batch_destroy(batch)
        for m in maps:
            m.close()


def test_barrier_timeout_is_reported_and_context_survives():
    """A grid-barrier wait that can never complete (one arrival that does not
    exist) gives up after its poll limit: the host sees TSDF_ERR_TIMEOUT and the
    GPU context stays usable."""
    from paper_2310_05766_gb300 import binding as b
    ws = _small_batch(2, seed=23)
    maps = [b.TsdfMap(w.params) for w in ws]
    pts = [torch.from_numpy(w.scans[0]).cuda() for w in ws]
    batch = b.tsdf_batch_create(2)
    b.tsdf_batch_set_option(batch, b.TSDF_BATCH_OPT_GRAPH, 0)
    b.tsdf_batch_set_option(batch, b.TSDF_BATCH_OPT_AUTOTUNE, 0)
    b.tsdf_batch_set_option(batch, b.TSDF_BATCH_OPT_SPIN_LIMIT, 20000)
    b.tsdf_batch_set_option(batch, b.TSDF_BATCH_OPT_TEST_MISSING_ARRIVALS, 1)
    b.tsdf_batch_integrate(batch, maps, pts, [w.poses[0] for w in ws])
    assert b.tsdf_batch_sync(batch) == b.TSDF_ERR_TIMEOUT
    b.tsdf_batch_destroy(batch)
    for m in maps:
        m.close()
    # the context still works: a fresh batch and fresh maps give exact results
    mb = _run_batch(b, ws)
    ms = _run_single(b, ws)
    _same(b, mb, ms)
    for m in mb + ms:
        m.close()
