"""tsdf_integrate_static: the allocation-free integration entry point.

Callers that cannot allocate device memory while running (a real-time loop
that reserves all memory at start-up, or a process whose device memory is
owned by another allocator) integrate into a grid they own, with all working
memory in a fixed device array inside the library. This file checks, through
the C ABI, that two calls in a row produce exactly the grid and counters that
the allocating path (tsdf_map_create + tsdf_integrate) produces and that the
oracle produces (pre-filled grid, ring-wrapping window origin, synchronous and
asynchronous calls), that an empty scan changes nothing, and that sizes beyond
the fixed array and malformed tensors are refused. It is named so that pytest
collects it last.
"""
import math

import numpy as np
import pytest

from paper_2310_05766_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class _DevView:
    """Wraps a raw device pointer for torch.as_tensor (CUDA array interface)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<u4", "data": (ptr, False), "version": 2}


def _two_scans():
    scene = synth.box_room_scene()
    dirs = synth.beam_directions(16, 360, -15.0, 15.0)
    poses = [(np.eye(3), np.zeros(3)), (synth.rot_zyx(0.3, 0.02, -0.01), np.array([0.35, -0.2, 0.05]))]
    out = []
    for i, (R, t) in enumerate(poses):
        pts = synth.make_scan(scene, R, t, dirs, 0.01, synth.SplitMix64(11 + i), r_max=20.0)
        out.append((pts, synth.pose12(R, t)))
    return out


def _params(reduce=0, flags=0):
    # 128 x 128 x 64 = 2^20 voxels (inside the fixed scratch limit) at 0.1 m:
    # the window covers the whole 10 x 10 x 3 m room
    return synth.params_dict((128, 128, 64), 0.1, 0.3, 64, synth.delta_z_for(30.0, 16), 0.3, 20.0, reduce,
                             (-64, -64, -32), flags=flags)


@pytest.mark.parametrize("reduce,flags", [(0, 0), (1, 0), (0, 3)])
def test_static_entry_matches_allocating_path(reduce, flags):
    from paper_2310_05766_gb300 import binding as b
    p = _params(reduce, flags)
    voxels = p["dims"][0] * p["dims"][1] * p["dims"][2]
    scans = _two_scans()
    # reference: the allocating entry points
    m = b.TsdfMap(p)
    ref_stats = []
    try:
        for pts, pose in scans:
            m.integrate(torch.from_numpy(pts).cuda(), pose)
            ref_stats.append(m.stats())
        torch.cuda.synchronize()
        ref = torch.as_tensor(_DevView(b.tsdf_grid_device_ptr(m.handle), voxels), device="cuda").cpu().numpy()
    finally:
        m.close()
    # the allocation-free entry point, two calls in a row into a caller-owned grid
    grid = torch.zeros(voxels, dtype=torch.int32, device="cuda")
    got_stats = []
    for pts, pose in scans:
        got_stats.append(b.tsdf_integrate_static(grid, p, torch.from_numpy(pts).cuda(), pts.shape[0], pose))
    got = grid.cpu().numpy().view(np.uint32)
    assert ref_stats[0]["hits"] > 50000 and ref_stats[1]["hits"] > 50000
    assert got_stats == ref_stats
    assert np.array_equal(got, ref)


def _grid_index(origin, dims):
    """Word index of every window voxel, shape (z, y, x), in the grid layout
    the header describes: ring slot s = g mod dims per axis, brick
    ((sz >> 3) * (dy / 8) + (sy >> 3)) * (dx / 8) + (sx >> 3), word
    brick * 512 + (sz & 7) * 64 + (sy & 7) * 8 + (sx & 7)."""
    g = [np.arange(origin[a], origin[a] + dims[a], dtype=np.int64) % dims[a] for a in range(3)]
    sz, sy, sx = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    brick = ((sz >> 3) * (dims[1] // 8) + (sy >> 3)) * (dims[0] // 8) + (sx >> 3)
    return brick * 512 + (sz & 7) * 64 + (sy & 7) * 8 + (sx & 7)


def _to_grid(v, w, origin, dims):
    out = np.zeros(dims[0] * dims[1] * dims[2], dtype=np.uint32)
    out[_grid_index(origin, dims)] = (v.astype(np.uint16).astype(np.uint32)
                                      | (w.astype(np.uint16).astype(np.uint32) << 16))
    return out


def _from_grid(grid, origin, dims):
    words = grid[_grid_index(origin, dims)]
    return (words & 0xFFFF).astype(np.uint16).view(np.int16), (words >> 16).astype(np.uint16).view(np.int16)


@pytest.mark.parametrize("reduce,flags,want_stats", [(0, 0, True), (1, 0, True), (0, 3, False), (0, 0, False)])
def test_static_entry_matches_oracle_prefilled_ring_origin(reduce, flags, want_stats):
    """Against the oracle directly: a pre-filled map, a window origin whose ring
    offset is non-zero on every axis, two scans in a row (without stats the
    calls are asynchronous, back to back on one stream, read after one
    synchronise)."""
    import oracle
    from paper_2310_05766_gb300 import binding as b
    origin = (-40, -72, -24)   # ring offsets 88, 56, 40 in a 128 x 128 x 64 window
    p = dict(_params(reduce, flags), origin=origin)
    dims = p["dims"]
    rng = np.random.default_rng(7 + reduce + 10 * flags)
    shape = (dims[2], dims[1], dims[0])
    w0 = np.where(rng.random(shape) < 0.3, rng.integers(1, 64, shape), 0).astype(np.int16)
    v0 = np.where(w0 > 0, rng.integers(-32767, 32768, shape), 0).astype(np.int16)
    scans = _two_scans()
    om = oracle.OracleMap(p)
    om.load_window(v0, w0)
    ref_stats = []
    for pts, pose in scans:
        om.integrate(pts, pose)
        ref_stats.append(om.stats())
    vo, wo = om.read()
    grid = torch.from_numpy(_to_grid(v0, w0, origin, dims).view(np.int32)).cuda()
    got_stats = []
    for pts, pose in scans:
        got_stats.append(b.tsdf_integrate_static(grid, p, torch.from_numpy(pts).cuda(), pts.shape[0], pose,
                                                 want_stats=want_stats))
    torch.cuda.synchronize()
    vg, wg = _from_grid(grid.cpu().numpy().view(np.uint32), origin, dims)
    assert ref_stats[0]["hits"] > 50000
    if want_stats:
        assert got_stats == ref_stats
    assert np.array_equal(wg, wo) and np.array_equal(vg, vo)


def test_static_entry_empty_scan_leaves_grid_unchanged():
    from paper_2310_05766_gb300 import binding as b
    p = _params()
    scans = _two_scans()
    grid = torch.zeros(128 * 128 * 64, dtype=torch.int32, device="cuda")
    b.tsdf_integrate_static(grid, p, torch.from_numpy(scans[0][0]).cuda(), scans[0][0].shape[0], scans[0][1])
    before = grid.clone()
    st = b.tsdf_integrate_static(grid, p, torch.zeros((0, 4), dtype=torch.float32, device="cuda"), 0, scans[0][1])
    assert st == dict(valid_rays=0, hits=0, touched=0)
    assert torch.equal(grid, before)


def test_static_entry_binding_rejects_bad_tensors():
    """The caller owns the grid, so the binding checks the tensors it is given."""
    from paper_2310_05766_gb300 import binding as b
    p = _params()
    pts, pose = _two_scans()[0]
    good_pts = torch.from_numpy(pts).cuda()
    small = torch.zeros(128 * 128 * 64 - 512, dtype=torch.int32, device="cuda")
    for grid, points in ((small, good_pts),
                         (torch.zeros(128 * 128 * 64, dtype=torch.int32, device="cuda"), good_pts.double()),
                         (torch.zeros(128 * 128 * 64, dtype=torch.float32, device="cuda"), good_pts),
                         (torch.zeros(128 * 128 * 64, dtype=torch.int64, device="cuda"), good_pts),
                         (torch.zeros(128 * 128 * 64, dtype=torch.int32, device="cuda"), good_pts[:, :3])):
        with pytest.raises(b.TsdfError) as e:
            b.tsdf_integrate_static(grid, p, points, pts.shape[0], pose)
        assert e.value.code == b.TSDF_ERR_INVALID
        assert not grid.any().item()
    with pytest.raises(b.TsdfError):   # n larger than the tensor
        b.tsdf_integrate_static(torch.zeros(128 * 128 * 64, dtype=torch.int32, device="cuda"), p, good_pts,
                                pts.shape[0] + 1, pose)


def test_static_entry_rejects_sizes_beyond_its_array():
    from paper_2310_05766_gb300 import binding as b
    scans = _two_scans()
    pts = torch.from_numpy(scans[0][0]).cuda()
    big = dict(_params(), dims=(256, 256, 64))          # 2^22 voxels > 2^21
    grid = torch.zeros(256 * 256 * 64, dtype=torch.int32, device="cuda")
    with pytest.raises(b.TsdfError) as e:
        b.tsdf_integrate_static(grid, big, pts, pts.shape[0], scans[0][1])
    assert e.value.code == b.TSDF_ERR_INVALID
    many = torch.zeros((b.TSDF_STATIC_MAX_POINTS + 1, 4), dtype=torch.float32, device="cuda")
    small_grid = torch.zeros(128 * 128 * 64, dtype=torch.int32, device="cuda")
    with pytest.raises(b.TsdfError) as e:
        b.tsdf_integrate_static(small_grid, _params(), many, many.shape[0], scans[0][1])
    assert e.value.code == b.TSDF_ERR_INVALID
    assert not small_grid.any().item()
