"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Every comparison is bit-exact on the whole value + weight window (integer
results; the float geometry is evaluated in the same IEEE order on both
sides), plus equality of the per-scan counters (valid rays, in-window
contributions, touched voxels).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_05766_gb300 import synth
from helpers import assert_same, run_gpu, run_oracle, workload_steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2310_05766_gb300 import binding
    binding.lib()
    yield


def both(params, steps, prefill=None, host=False, label="", options=None):
    g = run_gpu(params, steps, torch, prefill=prefill, host=host, options=options)
    o = run_oracle(params, steps, prefill=prefill)
    assert_same(g, o, label)
    return g, o


# ---------------------------------------------------------------- box room, one scan

@pytest.mark.parametrize("reduce", [0, 1])
def test_room_scan_exact(reduce):
    w = synth.workload_room(reduce=reduce)
    g, o = both(w.params, workload_steps(w), label=f"room reduce={reduce}")
    assert g[2][0]["hits"] > 300000 and g[2][0]["valid_rays"] == 5760


@pytest.mark.parametrize("reduce", [0, 1])
@pytest.mark.parametrize("merge,kpt,pdl,graph", [(1, 2, 1, 1), (0, 1, 1, 1), (0, 4, 1, 1), (1, 4, 0, 1), (0, 2, 0, 1),
                                                 (1, 1, 1, 1), (0, 4, 1, 0), (1, 2, 0, 0)])
def test_tuning_options_same_result(reduce, merge, kpt, pdl, graph):
    """Tuning options (warp match-merge, steps per thread, programmatic
    dependent launch, one graph launch per scan) change speed only: every
    setting is bit-identical to the oracle."""
    from paper_2310_05766_gb300 import binding as b
    opts = {b.TSDF_OPT_WARP_MERGE: merge, b.TSDF_OPT_STEPS_PER_THREAD: kpt, b.TSDF_OPT_PDL: pdl,
            b.TSDF_OPT_LAUNCH_GRAPH: graph}
    w = synth.workload_room(reduce=reduce)
    both(w.params, workload_steps(w), options=opts, label=f"room {opts}")
    w2 = synth.workload_outdoor(n_scans=2, reduce=reduce)
    both(w2.params, workload_steps(w2), options=opts, label=f"outdoor {opts}")
    p, steps = _rand_case(7)
    both(dict(p, reduce=reduce), steps, options=opts, label=f"random {opts}")


def test_launch_graph_and_plain_launches_exact():
    """The plain path's captured graph and four launches per scan (the default)
    both give the oracle's result, also when one map moves between them in
    the middle of a sequence: an option that rebuilds the graph, profiling
    (four launches), the graph turned off and on again, empty scans and scans
    of other sizes (the ray kernel's grid changes), and shifts."""
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_outdoor(n_scans=7)
    steps = workload_steps(w)
    sizes = [None, 1000, 0, 33, None, 4097, None]
    scans = [i for i, st in enumerate(steps) if st[0] == "scan"]
    for k, i in enumerate(scans):
        if sizes[k] is not None:
            steps[i] = ("scan", steps[i][1][:sizes[k]], steps[i][2])
    actions = {1: [(b.TSDF_OPT_STEPS_PER_THREAD, 2)], 3: ["profile_on"], 4: ["profile_off", (b.TSDF_OPT_LAUNCH_GRAPH, 0)],
               5: [(b.TSDF_OPT_LAUNCH_GRAPH, 1), (b.TSDF_OPT_STEPS_PER_THREAD, 4)]}
    m = b.TsdfMap(w.params)
    stats = []
    try:
        b.tsdf_set_option(m.handle, b.TSDF_OPT_LAUNCH_GRAPH, 1)
        k = 0
        for st in steps:
            if st[0] == "shift":
                m.shift(st[1])
                continue
            for act in actions.get(k, []):
                if act == "profile_on":
                    b.tsdf_profile_enable(m.handle, 1)
                elif act == "profile_off":
                    b.tsdf_profile_enable(m.handle, 0)
                else:
                    b.tsdf_set_option(m.handle, act[0], act[1])
            m.integrate(torch.from_numpy(np.ascontiguousarray(st[1])).cuda(), st[2])
            stats.append(m.stats())
            k += 1
        v, wt = m.read()
        g = (v, wt, stats, m.origin)
    finally:
        m.close()
    o = run_oracle(w.params, steps)
    assert_same(g, o, "graph / plain launches")
    assert stats[2]["hits"] == 0 and stats[0]["hits"] > 1000000


def test_invalid_option_rejected():
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_room()
    m = b.TsdfMap(w.params)
    try:
        for opt, val in [(b.TSDF_OPT_STEPS_PER_THREAD, 3), (b.TSDF_OPT_WARP_MERGE, 2), (b.TSDF_OPT_PDL, -1),
                         (b.TSDF_OPT_LAUNCH_GRAPH, 2), (99, 0)]:
            with pytest.raises(b.TsdfError):
                b.tsdf_set_option(m.handle, opt, val)
    finally:
        m.close()


def test_room_scan_into_prefilled_map():
    w = synth.workload_room()
    rng = np.random.default_rng(1)
    d = w.params["dims"]
    v0 = rng.integers(-32767, 32768, size=(d[2], d[1], d[0])).astype(np.int16)
    w0 = rng.integers(0, w.params["w_max"] + 1, size=v0.shape).astype(np.int16)
    steps = workload_steps(w) + [("scan", w.scans[0], w.poses[0])]
    both(w.params, steps, prefill=(v0, w0), label="prefilled")


def test_room_host_points_path():
    w = synth.workload_room()
    both(w.params, workload_steps(w), host=True, label="host points")


@pytest.mark.parametrize("zero_copy", [1, 0])
def test_host_pinned_points_path(zero_copy):
    """Pinned host points: read in place by the rays kernel (zero copy) or
    staged; both exact, counters read back through the mapped copy. A pinned
    buffer that is not 16-byte aligned takes the staging copy."""
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_outdoor(n_scans=3)
    steps = workload_steps(w)
    m = b.TsdfMap(w.params)
    stats = []
    try:
        b.tsdf_set_option(m.handle, b.TSDF_OPT_HOST_ZERO_COPY, zero_copy)
        for k, st in enumerate(steps):
            if st[0] == "shift":
                m.shift(st[1])
                continue
            n = st[1].shape[0]
            if k % 2 == 0:
                pinned = torch.from_numpy(np.ascontiguousarray(st[1], np.float32)).pin_memory()
                m.integrate_host(pinned, st[2])
            else:   # 4 bytes past a 16-byte boundary
                buf = torch.empty(4 * n + 1, dtype=torch.float32).pin_memory()
                buf[1:] = torch.from_numpy(np.ascontiguousarray(st[1], np.float32).reshape(-1))
                b.tsdf_integrate_host(m.handle, buf.data_ptr() + 4, n, st[2])
            stats.append(m.stats())   # synchronises: the buffers may go now
        v, wt = m.read()
    finally:
        m.close()
    vo, wo, so, _ = run_oracle(w.params, steps)
    assert np.array_equal(v, vo) and np.array_equal(wt, wo)
    assert stats == so


def test_point_order_does_not_matter():
    w = synth.workload_room()
    perm = np.random.default_rng(2).permutation(w.scans[0].shape[0])
    a = run_gpu(w.params, [("scan", w.scans[0], w.poses[0])], torch)
    b = run_gpu(w.params, [("scan", w.scans[0][perm], w.poses[0])], torch)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


# ---------------------------------------------------------------- random small cases

def _rand_case(seed):
    rng = np.random.default_rng(1000 + seed)
    dims = tuple(int(x) for x in rng.choice([8, 16, 32, 64], size=3))
    vs = float(rng.choice([0.05, 0.0625, 0.08, 0.1]))
    tau = float(vs * rng.uniform(1.0, 5.0))
    origin = tuple(int(8 * rng.integers(-8, 4)) for _ in range(3))
    dz = float(rng.choice([0.0, 0.01, 0.05, 0.2]))
    reduce = int(rng.integers(0, 2))
    w_max = int(rng.integers(1, 40))
    p = synth.params_dict(dims, vs, tau, w_max, dz, 0.05, 6.0, reduce, origin)
    centre = np.array([(origin[a] + dims[a] / 2) * vs for a in range(3)])
    steps = []
    cur = origin
    for s in range(int(rng.integers(1, 5))):
        n = int(rng.choice([1, 31, 33, 255, 257, 1000, 3001]))
        pts = np.zeros((n, 4), np.float32)
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pts[:, :3] = d * rng.uniform(0.02, 2.5, (n, 1))
        if n > 4:
            pts[rng.integers(0, n, n // 8), rng.integers(0, 3)] = np.nan
        R = synth.rot_zyx(*rng.uniform(-math.pi, math.pi, 3))
        t = centre + rng.uniform(-0.5, 0.5, 3)
        steps.append(("scan", pts, synth.pose12(R, t)))
        if rng.uniform() < 0.5:
            cur = tuple(int(cur[a] + 8 * rng.integers(-2, 3)) for a in range(3))
            steps.append(("shift", cur))
    return p, steps


@pytest.mark.parametrize("seed", range(40))
def test_random_small_exact(seed):
    p, steps = _rand_case(seed)
    both(p, steps, label=f"random seed {seed}")


# ---------------------------------------------------------------- sort reduction

def _sort_opts(b, kpt=4, cap=0):
    return {b.TSDF_OPT_REDUCTION: b.TSDF_REDUCTION_SORT, b.TSDF_OPT_STEPS_PER_THREAD: kpt,
            b.TSDF_OPT_SORT_CAPACITY: cap}


@pytest.mark.parametrize("reduce", [0, 1])
@pytest.mark.parametrize("kpt", [4, 2, 1])
def test_sort_reduction_exact(reduce, kpt):
    """The counting-sort reduction gives the same maps and counters as the
    oracle (and so as the atomic reduction): room, two outdoor scans with a
    shift, a random case with shifts."""
    from paper_2310_05766_gb300 import binding as b
    opts = _sort_opts(b, kpt)
    w = synth.workload_room(reduce=reduce)
    both(w.params, workload_steps(w) + [("scan", w.scans[0], w.poses[0])], options=opts, label=f"room sort {kpt}")
    w2 = synth.workload_outdoor(n_scans=12, reduce=reduce)
    both(w2.params, workload_steps(w2)[:4], options=opts, label=f"outdoor sort {kpt}")
    p, steps = _rand_case(7)
    both(dict(p, reduce=reduce), steps, options=opts, label=f"random sort {kpt}")


@pytest.mark.parametrize("cap", [1024, 65536, 250000])
@pytest.mark.parametrize("reduce", [0, 1])
def test_sort_reduction_overflow_exact(cap, reduce):
    """Pair capacities far below the scan's samples: the samples beyond it go
    to the accumulator atomics and are merged per brick; still exact."""
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_room(reduce=reduce)
    steps = workload_steps(w) + [("scan", w.scans[0], w.poses[0])]
    g, o = both(w.params, steps, options=_sort_opts(b, 4, cap), label=f"room sort cap {cap}")
    assert g[2][0]["hits"] > cap


@pytest.mark.parametrize("seed", range(16))
def test_random_small_sort_exact(seed):
    from paper_2310_05766_gb300 import binding as b
    p, steps = _rand_case(seed)
    both(dict(p, flags=seed % 4), steps, options=_sort_opts(b, [4, 2, 1][seed % 3], [0, 0, 1024, 4096][seed % 4]),
         label=f"random sort seed {seed}")


def test_sort_reduction_edge_cases():
    """Empty and all-invalid scans, many rays through the same voxels, the
    weight cap and a switch between reductions on one map."""
    from paper_2310_05766_gb300 import binding as b
    p = _edge_params()
    rng = np.random.default_rng(21)
    empty = np.zeros((0, 4), np.float32)
    nan = np.full((100, 4), np.nan, np.float32)
    pose = synth.pose12(np.eye(3), np.zeros(3))
    same = np.tile(np.array([[1.0, 0.2, 0.1, 0.0]], np.float32), (4096, 1))
    pts = np.zeros((2000, 4), np.float32)
    d = rng.normal(size=(2000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts[:, :3] = d * rng.uniform(0.3, 1.5, (2000, 1))
    steps = [("scan", empty, pose), ("scan", nan, pose), ("scan", same, pose), ("scan", pts, pose)]
    steps += [("scan", pts, pose)] * 3
    for reduce in (0, 1):
        both(dict(p, reduce=reduce, w_max=3), steps, options=_sort_opts(b), label=f"sort edges {reduce}")
    # switching the reduction between scans of one map
    m = b.TsdfMap(p)
    try:
        for i, st in enumerate(steps[2:]):
            b.tsdf_set_option(m.handle, b.TSDF_OPT_REDUCTION, i % 3)
            m.integrate(torch.from_numpy(st[1]).cuda(), st[2])
        vg, wg = m.read()
    finally:
        m.close()
    vo, wo, _, _ = run_oracle(p, steps[2:])
    assert np.array_equal(vg, vo) and np.array_equal(wg, wo)


def test_sort_options_rejected():
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_room()
    m = b.TsdfMap(w.params)
    try:
        for opt, val in [(b.TSDF_OPT_REDUCTION, 4), (b.TSDF_OPT_REDUCTION, -1), (b.TSDF_OPT_SORT_CAPACITY, 5),
                         (b.TSDF_OPT_SORT_CAPACITY, (1 << 28) + 1), (b.TSDF_OPT_POOL_BRICKS, 63),
                         (b.TSDF_OPT_POOL_BRICKS, 1 << 30)]:
            with pytest.raises(b.TsdfError):
                b.tsdf_set_option(m.handle, opt, val)
    finally:
        m.close()


def test_auto_reduction_decides_and_stays_exact():
    """TSDF_REDUCTION_AUTO runs both reductions on the first calls (each
    once untimed, then timed), keeps the faster one, and every scan on the way
    is exact."""
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_outdoor(n_scans=12)
    steps = workload_steps(w) + [("scan", w.scans[i], w.poses[i]) for i in range(11, 0, -1)]
    m = b.TsdfMap(w.params)
    try:
        b.tsdf_set_option(m.handle, b.TSDF_OPT_REDUCTION, b.TSDF_REDUCTION_AUTO)
        assert b.tsdf_get_reduction(m.handle) == b.TSDF_REDUCTION_AUTO
        stats = []
        for st in steps:
            if st[0] == "shift":
                m.shift(st[1])
                continue
            m.integrate(torch.from_numpy(st[1]).cuda(), st[2])
            stats.append(m.stats())
        chosen = b.tsdf_get_reduction(m.handle)
        v, wt = m.read()
    finally:
        m.close()
    assert chosen in (b.TSDF_REDUCTION_ATOMIC, b.TSDF_REDUCTION_SORT, b.TSDF_REDUCTION_POOL)
    vo, wo, so, _ = run_oracle(w.params, steps)
    assert np.array_equal(v, vo) and np.array_equal(wt, wo) and stats == so


# ---------------------------------------------------------------- pool reduction (sparse accumulator)

def _pool_opts(b, kpt=4, bricks=0):
    return {b.TSDF_OPT_REDUCTION: b.TSDF_REDUCTION_POOL, b.TSDF_OPT_STEPS_PER_THREAD: kpt,
            b.TSDF_OPT_POOL_BRICKS: bricks}


@pytest.mark.parametrize("reduce", [0, 1])
@pytest.mark.parametrize("kpt", [4, 1])
def test_pool_reduction_exact(reduce, kpt):
    """Per-scan accumulators in pooled bricks claimed on first touch: the
    same maps and counters as the oracle (room twice, outdoor prefix with a
    shift, a random case with shifts)."""
    from paper_2310_05766_gb300 import binding as b
    opts = _pool_opts(b, kpt)
    w = synth.workload_room(reduce=reduce)
    both(w.params, workload_steps(w) + [("scan", w.scans[0], w.poses[0])], options=opts, label=f"room pool {kpt}")
    w2 = synth.workload_outdoor(n_scans=12, reduce=reduce)
    both(w2.params, workload_steps(w2)[:5], options=opts, label=f"outdoor pool {kpt}")
    p, steps = _rand_case(9)
    both(dict(p, reduce=reduce), steps, options=opts, label=f"random pool {kpt}")


@pytest.mark.parametrize("seed", range(12))
def test_random_small_pool_exact(seed):
    from paper_2310_05766_gb300 import binding as b
    p, steps = _rand_case(seed)
    nb = (p["dims"][0] // 8) * (p["dims"][1] // 8) * (p["dims"][2] // 8)
    # a pool of exactly the window's bricks, or the default (also all of them for these small windows)
    both(dict(p, flags=seed % 4), steps, options=_pool_opts(b, [4, 2, 1][seed % 3], nb if seed % 2 and nb >= 64 else 0),
         label=f"random pool seed {seed}")


def test_pool_full_drops_scan_and_recovers():
    """A pool smaller than the scan's touched bricks: the scan is dropped
    whole (TSDF_ERR_CAPACITY, map unchanged); with a large enough pool the
    same map then integrates it exactly."""
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_room()
    m = b.TsdfMap(w.params)
    try:
        pts = torch.from_numpy(w.scans[0]).cuda()
        m.integrate(pts, w.poses[0])                 # atomic reduction first
        v0, w0 = m.read()
        b.tsdf_set_option(m.handle, b.TSDF_OPT_REDUCTION, b.TSDF_REDUCTION_POOL)
        b.tsdf_set_option(m.handle, b.TSDF_OPT_POOL_BRICKS, 64)
        m.integrate(pts, w.poses[0])
        with pytest.raises(b.TsdfError) as ei:
            m.stats()
        assert ei.value.code == b.TSDF_ERR_CAPACITY
        v1, w1 = m.read()
        assert np.array_equal(v0, v1) and np.array_equal(w0, w1)
        b.tsdf_set_option(m.handle, b.TSDF_OPT_POOL_BRICKS, 0)
        m.integrate(pts, w.poses[0])
        st = m.stats()
        v2, w2 = m.read()
    finally:
        m.close()
    vo, wo, so, _ = run_oracle(w.params, [("scan", w.scans[0], w.poses[0])] * 2)
    assert np.array_equal(v2, vo) and np.array_equal(w2, wo) and st == so[1]


def test_pool_map_holds_no_dense_accumulator():
    """A map used only with the pool reduction never allocates the 8 B/voxel
    accumulator; switching to the atomic reduction allocates it, and all
    three reductions interleave on one map with exact results."""
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_outdoor(n_scans=4)
    p = w.params
    voxels = p["dims"][0] * p["dims"][1] * p["dims"][2]
    m = b.TsdfMap(p)
    try:
        b.tsdf_set_option(m.handle, b.TSDF_OPT_REDUCTION, b.TSDF_REDUCTION_POOL)
        steps = workload_steps(w)
        for i, st in enumerate(steps):
            if st[0] == "shift":
                m.shift(st[1])
                continue
            if i == 2:
                pool_bytes = b.tsdf_map_device_bytes(m.handle)
                assert pool_bytes < voxels * 4 + voxels * 8 // 2, pool_bytes
                b.tsdf_set_option(m.handle, b.TSDF_OPT_REDUCTION, b.TSDF_REDUCTION_ATOMIC)
            if i == 3:
                b.tsdf_set_option(m.handle, b.TSDF_OPT_REDUCTION, b.TSDF_REDUCTION_SORT)
            m.integrate(torch.from_numpy(st[1]).cuda(), st[2])
            m.stats()
        assert b.tsdf_map_device_bytes(m.handle) >= voxels * 12
        v, wt = m.read()
    finally:
        m.close()
    vo, wo, _, _ = run_oracle(p, steps)
    assert np.array_equal(v, vo) and np.array_equal(wt, wo)


# ---------------------------------------------------------------- alternative readings (map flags)

@pytest.mark.parametrize("flags", [1, 2, 3])
@pytest.mark.parametrize("reduce", [0, 1])
def test_room_flags_exact(flags, reduce):
    """Step-valued fill (flag 1) and one observation per scan (flag 2): two
    scans (the second onto a map with weights) bit-exact against the oracle."""
    w = synth.workload_room(reduce=reduce)
    p = dict(w.params, flags=flags)
    steps = workload_steps(w) + [("scan", w.scans[0], w.poses[0])]
    g, o = both(p, steps, label=f"room flags={flags} reduce={reduce}")
    assert g[2][0]["hits"] > 300000


@pytest.mark.parametrize("flags", [1, 2, 3])
def test_flags_with_tuning_options(flags):
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_outdoor(n_scans=2)
    for merge, kpt in [(1, 2), (0, 1)]:
        opts = {b.TSDF_OPT_WARP_MERGE: merge, b.TSDF_OPT_STEPS_PER_THREAD: kpt}
        both(dict(w.params, flags=flags), workload_steps(w), options=opts, label=f"outdoor flags={flags} {opts}")


@pytest.mark.parametrize("seed", range(12))
def test_random_small_flags_exact(seed):
    p, steps = _rand_case(seed)
    both(dict(p, flags=seed % 3 + 1), steps, label=f"random seed {seed} flags {seed % 3 + 1}")


def test_unknown_flag_bits_rejected():
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_room()
    for fl in (4, 8, -1):
        with pytest.raises(b.TsdfError):
            b.TsdfMap(dict(w.params, flags=fl))


# ---------------------------------------------------------------- edge cases

def _edge_params(**kw):
    base = synth.params_dict((32, 32, 32), 0.1, 0.3, 64, 0.05, 0.5, 2.0, 0, (-16, -16, -16))
    base.update(kw)
    return base


def test_empty_scan_and_all_invalid():
    p = _edge_params()
    pose = synth.pose12(np.eye(3), np.zeros(3))
    nan = np.full((100, 4), np.nan, np.float32)
    zeros = np.zeros((64, 4), np.float32)
    far = np.tile(np.array([[5.0, 0, 0, 0]], np.float32), (40, 1))   # beyond r_max
    g, o = both(p, [("scan", np.zeros((0, 4), np.float32), pose), ("scan", nan, pose), ("scan", zeros, pose),
                    ("scan", far, pose)], label="empty/invalid")
    assert all(s == dict(valid_rays=0, hits=0, touched=0) for s in g[2])
    assert not g[0].any() and not g[1].any()


def test_range_limits_and_degenerate_fill():
    p = _edge_params()
    pose = synth.pose12(np.eye(3), np.zeros(3))
    pts = np.array([[0.5, 0, 0, 0], [2.0, 0, 0, 0], [0, 0, 1.5, 0], [0, 0, -1.2, 0], [0.49999, 0, 0, 0],
                    [2.0001, 0, 0, 0], [1.0, 1.0, 0.5, 0]], np.float32)
    g, o = both(p, [("scan", pts, pose)], label="limits")
    assert g[2][0]["valid_rays"] == 5


def test_fill_disabled_and_tiny_window():
    p = _edge_params(dims=(8, 8, 8), origin=(-8, 0, -8), delta_z=0.0)
    rng = np.random.default_rng(3)
    pts = np.zeros((500, 4), np.float32)
    pts[:, :3] = rng.uniform(-1.2, 1.2, (500, 3))
    both(p, [("scan", pts, synth.pose12(synth.rot_zyx(0.3, 0.2, 0.1), np.array([0.0, 0.4, 0.0])))], label="tiny")


@pytest.mark.parametrize("rlo, rhi", [(0.5, 2.0), (0.5, 1.2), (1.3, 2.0)])
def test_heavy_and_light_rays(rlo, rhi):
    """The plain path orders its ray list by fill size (rays with delta_z r >=
    voxel size first): mixed, light-only and heavy-only scans, with both parts
    of the list ending inside a 32-ray block."""
    p = _edge_params(delta_z=0.08)   # heavy from r = 1.25 m
    rng = np.random.default_rng(11)
    for n in (1, 37, 1001):
        pts = np.zeros((n, 4), np.float32)
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pts[:, :3] = d * rng.uniform(rlo, rhi, (n, 1))
        pose = synth.pose12(synth.rot_zyx(0.4, 0.1, -0.2), np.array([0.05, -0.1, 0.02]))
        both(p, [("scan", pts, pose), ("scan", pts[::-1].copy(), pose)], label=f"split n={n} r=[{rlo},{rhi}]")


def test_weight_cap_reached():
    p = _edge_params(w_max=3)
    pose = synth.pose12(np.eye(3), np.zeros(3))
    pts = np.tile(np.array([[1.03, 0.21, 0.05, 0]], np.float32), (20, 1))
    g, o = both(p, [("scan", pts, pose)] * 3, label="cap")
    assert g[1].max() == 3


def test_many_hits_on_one_voxel():
    """Hundreds of rays through the same voxels: heavy intra-warp and inter-warp merging."""
    p = _edge_params(delta_z=0.3)
    pose = synth.pose12(np.eye(3), np.array([0.01, 0.02, 0.03]))
    rng = np.random.default_rng(5)
    pts = np.tile(np.array([[1.2, 0.3, 0.1, 0]], np.float32), (4096, 1))
    pts[:, :3] += rng.normal(scale=0.002, size=(4096, 3)).astype(np.float32)
    for reduce in (0, 1):
        both(dict(p, reduce=reduce), [("scan", pts, pose)], label=f"dense reduce={reduce}")


# ---------------------------------------------------------------- shift

def test_shift_sequence_exact():
    w = synth.workload_room()
    p = dict(w.params, dims=(128, 128, 64), origin=(-64, -64, -32))
    o = p["origin"]
    steps = [("scan", w.scans[0], w.poses[0])]
    for d in [(8, 0, 0), (8, -16, 0), (0, 0, 8), (-64, 40, -8), (512, 0, 0), (0, 0, 0), (24, 24, 8)]:
        steps.append(("shift", (o[0] + d[0], o[1] + d[1], o[2] + d[2])))
        steps.append(("scan", w.scans[0], w.poses[0]))
    both(p, steps, label="shift sequence")


def test_shift_unshift_identity_gpu():
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_room()
    m = b.TsdfMap(w.params)
    try:
        m.integrate(torch.from_numpy(w.scans[0]).cuda(), w.poses[0])
        v0, w0 = m.read()
        o = w.params["origin"]
        m.shift((o[0] + 40, o[1] - 16, o[2] + 8))
        m.shift((o[0] + 4096, o[1], o[2]))
        m.shift(o)
        v1, w1 = m.read()
        assert np.array_equal(v0, v1) and np.array_equal(w0, w1)
    finally:
        m.close()


# ---------------------------------------------------------------- full-size workloads

def test_outdoor_sequence_prefix_exact():
    """OS1-128-shaped outdoor sequence at full size (512 x 512 x 128 at 0.064 m):
    the first 12 scans, including the first 1 m re-centring shift."""
    w = synth.workload_outdoor(n_scans=12)
    steps = workload_steps(w)
    assert any(s[0] == "shift" for s in steps)
    g, o = both(w.params, steps, label="outdoor prefix")
    assert min(s["hits"] for s in g[2]) > 1_000_000


def test_store_over_several_allocations():
    """A 64^3 window moved by its own size 26 times (512 chunks stored per
    shift, over 13 k in all: store segments from three growing allocations)
    with a scan at every position, then walked back, reading every stored
    chunk again; compared with the oracle throughout."""
    p = synth.params_dict((64, 64, 64), 0.1, 0.3, 64, 0.05, 0.3, 3.0, 0, (0, 0, 0))
    rng = np.random.default_rng(21)
    pts = np.zeros((3000, 4), np.float32)
    d = rng.normal(size=(3000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts[:, :3] = d * rng.uniform(0.5, 2.8, (3000, 1))
    steps = []
    checks = []   # walk-back positions whose chunks sit in the third, second and first allocation
    xs = list(range(0, 27)) + list(range(25, -1, -1))
    for k, xi in enumerate(xs):
        origin = (64 * xi, 0, 0)
        if k > 0:
            steps.append(("shift", origin))
        t = np.array([(origin[0] + 32) * 0.1, 3.2, 3.2])
        steps.append(("scan", pts, synth.pose12(synth.rot_zyx(0.1 * k, 0.0, 0.0), t)))
        if k > 26 and xi in (24, 20, 0):
            checks.append((xi, len(steps)))
    for xi, n in checks:
        both(p, steps[:n], label=f"store over several allocations, back at x = {64 * xi}")


def test_corridor_prefix_exact():
    """High-resolution corridor at full size (1024 x 1024 x 256 at 0.02 m): two
    scans, a 24-voxel shift along x, one more scan."""
    w = synth.workload_corridor(n_scans=3)
    o = w.params["origin"]
    steps = [("scan", w.scans[0], w.poses[0]), ("scan", w.scans[1], w.poses[1]),
             ("shift", (o[0] + 24, o[1], o[2])), ("scan", w.scans[2], w.poses[2])]
    g, o2 = both(w.params, steps, label="corridor prefix")
    assert min(s["hits"] for s in g[2]) > 3_000_000


def test_maximum_window_size():
    """A 2048 x 2048 x 512 window (2^31 voxels, the largest accepted): the box-room
    scan gives, inside the room's 256 x 256 x 64 sub-box, exactly the oracle's
    result for a window of that sub-box."""
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_room()
    pbig = dict(w.params, dims=(2048, 2048, 512), origin=(-1024, -1024, -256))
    m = b.TsdfMap(pbig)
    try:
        m.integrate(torch.from_numpy(w.scans[0]).cuda(), w.poses[0])
        lo = w.params["origin"]
        hi = tuple(lo[a] + w.params["dims"][a] for a in range(3))
        vg, wg = m.read(lo, hi)
    finally:
        m.close()
    om = oracle.OracleMap(w.params)
    om.integrate(w.scans[0], w.poses[0])
    vo, wo = om.read()
    assert np.array_equal(vg, vo) and np.array_equal(wg, wo)


# ---------------------------------------------------------------- argument errors on the GPU path

def test_invalid_arguments_leave_map_unchanged():
    from paper_2310_05766_gb300 import binding as b
    w = synth.workload_room()
    m = b.TsdfMap(w.params)
    try:
        pts = torch.from_numpy(w.scans[0]).cuda()
        m.integrate(pts, w.poses[0])
        v0, w0 = m.read()
        raw = pts.data_ptr()
        with pytest.raises(b.TsdfError) as e:
            b.tsdf_integrate(m.handle, raw + 4, 10, w.poses[0])   # misaligned
        assert e.value.code == b.TSDF_ERR_INVALID
        with pytest.raises(b.TsdfError):
            b.tsdf_integrate(m.handle, raw, b.TSDF_MAX_POINTS + 1, w.poses[0])
        bad_pose = w.poses[0].copy()
        bad_pose[3] = np.nan
        with pytest.raises(b.TsdfError):
            b.tsdf_integrate(m.handle, raw, 10, bad_pose)
        with pytest.raises(b.TsdfError):
            m.shift((3, 0, 0))
        with pytest.raises(b.TsdfError):
            m.read((0, 0, 0), (10**6, 1, 1))
        v1, w1 = m.read()
        assert np.array_equal(v0, v1) and np.array_equal(w0, w1)
    finally:
        m.close()


def test_write_read_roundtrip():
    from paper_2310_05766_gb300 import binding as b
    p = _edge_params()
    rng = np.random.default_rng(7)
    v = rng.integers(-32767, 32768, size=(32, 32, 32)).astype(np.int16)
    wt = rng.integers(0, 65, size=(32, 32, 32)).astype(np.int16)
    m = b.TsdfMap(p)
    try:
        m.write(v, wt)
        v1, w1 = m.read()
        assert np.array_equal(v, v1) and np.array_equal(wt, w1)
        lo = (-10, -3, 0)
        hi = (5, 7, 9)
        vs, ws = m.read(lo, hi)
        o = p["origin"]
        assert np.array_equal(vs, v[lo[2] - o[2]:hi[2] - o[2], lo[1] - o[1]:hi[1] - o[1], lo[0] - o[0]:hi[0] - o[0]])
        bad = wt.copy()
        bad[0, 0, 0] = 65
        with pytest.raises(b.TsdfError):
            m.write(v, bad)
    finally:
        m.close()


def test_packed_count_at_the_documented_maximum():
    """One voxel at the largest per-scan count the packed accumulator must hold.

    A ray whose march lattice puts four of its nine samples (tau = voxel size,
    fill J = 1) into voxel (5, 0, 12) -- the most one ray can, by the lattice
    argument of TSDF_MAX_POINTS -- repeated TSDF_MAX_POINTS times: the voxel's
    count is 4 (2^22 - 1) = 2^24 - 4, just inside the 24-bit count field of
    the packed word. The grid and counters must equal the oracle's (int64
    maps, no packing)."""
    import oracle
    from paper_2310_05766_gb300 import binding as b
    pt = np.array([[1.5753395557403564, 0.6343674659729004, 0.46042734384536743, 0.0]], np.float32)
    pose = np.array([-0.025146624073386192, 0.975757896900177, 0.2174031287431717, 0.0,
                     -0.1916240155696869, -0.21814407408237457, 0.9569187164306641, 0.0,
                     0.9811462163925171, -0.01759638637304306, 0.19246424734592438, 0.0], np.float32)
    p = synth.params_dict((8, 8, 8), 0.125, 0.125, 32767, 0.08914640378552456, 0.0, 100.0, 0, (0, 0, 8))
    g, q, ray = oracle.hits(p, pt, pose)
    voxels, counts = np.unique(g, axis=0, return_counts=True)
    assert len(g) == 9 and counts.max() == 4 and tuple(voxels[counts.argmax()]) == (5, 0, 12)
    assert b.TSDF_MAX_POINTS * 4 == (1 << 24) - 4
    n = b.TSDF_MAX_POINTS
    pts = np.repeat(pt, n, axis=0)
    steps = [("scan", pts, pose)]
    gpu = run_gpu(p, steps, torch)
    orc = run_oracle(p, steps)
    assert_same(gpu, orc, "maximum count")
    assert orc[2][0]["hits"] == 6 * n          # three of the nine samples fall outside the window (y = -1)
    assert orc[1][12 - 8, 0, 5] == 32767       # weight capped by Eq. 2; the count itself was 2^24 - 4
