"""tsdf_integrate_static: the allocation-free integration entry point.

Callers that cannot allocate device memory while running (a real-time loop
that reserves all memory at start-up, or a process whose device memory is
owned by another allocator) integrate into a grid they own, with all working
memory in a fixed device array inside the library. This file checks, through
the C ABI, that two calls in a row produce exactly the grid and counters that
the allocating path (tsdf_map_create + tsdf_integrate) produces, and that sizes
beyond the fixed array are refused. It is named so that pytest collects it
last.
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
