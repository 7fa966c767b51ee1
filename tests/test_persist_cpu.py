"""Map files on the host side: the loader rejects files that are missing,
foreign, truncated or carry invalid parameters before touching the device, and
the oracle's global map (window + chunk store) is unchanged by shifts."""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_2310_05766_gb300 import synth


def _header(params, count, magic=b"TSDFMAP1", version=1):
    from paper_2310_05766_gb300 import binding as b
    prm = b.make_params(params)
    h = bytearray(b.FILE_HEADER_BYTES)
    h[0:8] = magic
    h[8:12] = np.uint32(version).tobytes()
    h[12:16] = np.uint32(b.FILE_HEADER_BYTES).tobytes()
    h[16:16 + ctypes.sizeof(prm)] = bytes(prm)
    h[88:96] = np.int64(count).tobytes()
    return bytes(h)


def test_loader_rejects_bad_files_without_gpu(tmp_path):
    from paper_2310_05766_gb300 import binding as b
    p = synth.params_dict((64, 64, 64), 0.1, 0.3, 64, 0.0, 0.1, 10.0, 0, (-32, -32, -32))
    rec = bytes(b.FILE_RECORD_BYTES)
    cases = {
        "missing": None,
        "magic": _header(p, 0, magic=b"NOTAMAP!"),
        "version": _header(p, 0, version=2),
        "truncated": _header(p, 2) + rec,
        "longer": _header(p, 0) + rec,
        "params": _header(dict(p, dims=(60, 64, 64)), 0),
        "origin": _header(dict(p, origin=(-31, -32, -32)), 0),
        "short": b"TSDFMAP1",
    }
    for name, content in cases.items():
        path = str(tmp_path / f"{name}.tsdf")
        if content is not None:
            with open(path, "wb") as f:
                f.write(content)
        h = ctypes.c_void_p()
        rc = b.lib().tsdf_map_load(os.fsencode(path), ctypes.byref(h), None)
        assert rc == b.TSDF_ERR_IO, name
        assert h.value is None
    assert b.lib().tsdf_map_load(None, None, None) == b.TSDF_ERR_INVALID
    assert b.tsdf_error_string(b.TSDF_ERR_IO) == "file error or not a map file"


def test_file_layout_constants():
    from paper_2310_05766_gb300 import binding as b
    assert ctypes.sizeof(b.tsdf_params) == 72
    assert b.FILE_HEADER_BYTES == 8 + 4 + 4 + 72 + 8 + 32
    assert b.FILE_RECORD_BYTES == 3 * 8 + 512 * 4


def test_oracle_global_map_invariant_under_shifts():
    """Shifting the window moves chunks between the window and the store but
    leaves the global map unchanged, chunk for chunk; integrating a scan after
    the shifts matches integrating it before them."""
    w = synth.workload_room(seed=4)
    p = dict(w.params, dims=(128, 128, 64), origin=(-64, -64, -32), voxel_size=0.1)
    m = oracle.OracleMap(p)
    m.integrate(w.scans[0], w.poses[0])
    ref = m.global_chunks()
    assert len(ref) > 400
    for o in [(-48, -64, -32), (40, 8, -8), (-200, 0, 0), (-64, -64, -32)]:
        m.shift(o)
        got = m.global_chunks()
        assert got.keys() == ref.keys()
        for k in ref:
            assert np.array_equal(got[k][0], ref[k][0]) and np.array_equal(got[k][1], ref[k][1])
    m.shift((-40, -72, -24))
    m.integrate(w.scans[0], w.poses[0])
    m2 = oracle.OracleMap(p)
    m2.integrate(w.scans[0], w.poses[0])
    m2.shift((-40, -72, -24))
    m2.integrate(w.scans[0], w.poses[0])
    a, b2 = m.global_chunks(), m2.global_chunks()
    assert a.keys() == b2.keys()
    assert all(np.array_equal(a[k][0], b2[k][0]) and np.array_equal(a[k][1], b2[k][1]) for k in a)
