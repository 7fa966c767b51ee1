"""Shared helpers for the GPU parity tests: run the same sequence of scans and
shifts through the CUDA library and through the oracle, and compare grids."""
import numpy as np

import oracle


def run_gpu(params, steps, torch, prefill=None, host=False, options=None):
    """steps: list of ("scan", points(N,4) float32, pose[12]) or ("shift", origin3).
    options: {tsdf option id: value} applied after creation."""
    from paper_2310_05766_gb300 import binding as b
    m = b.TsdfMap(params)
    stats = []
    try:
        for opt, val in (options or {}).items():
            b.tsdf_set_option(m.handle, opt, val)
        if prefill is not None:
            m.write(prefill[0], prefill[1])
        for st in steps:
            if st[0] == "scan":
                if host:
                    m.integrate_host(np.ascontiguousarray(st[1], np.float32), st[2])
                else:
                    pts = torch.from_numpy(np.ascontiguousarray(st[1], np.float32)).cuda()
                    m.integrate(pts, st[2])
                stats.append(m.stats())
            else:
                m.shift(st[1])
        v, w = m.read()
        origin = m.origin
    finally:
        m.close()
    return v, w, stats, origin


def run_oracle(params, steps, prefill=None):
    m = oracle.OracleMap(params)
    stats = []
    if prefill is not None:
        m.load_window(prefill[0], prefill[1])
    for st in steps:
        if st[0] == "scan":
            m.integrate(st[1], st[2])
            stats.append(m.stats())
        else:
            m.shift(st[1])
    v, w = m.read()
    return v, w, stats, m.origin


def assert_same(gpu, orc, label=""):
    vg, wg, sg, og = gpu
    vo, wo, so, oo = orc
    assert og == oo, (label, og, oo)
    if not (np.array_equal(vg, vo) and np.array_equal(wg, wo)):
        dv = np.argwhere((vg != vo) | (wg != wo))
        z, y, x = dv[0]
        raise AssertionError(f"{label}: {len(dv)} voxels differ; first at (z,y,x)={tuple(dv[0])}: "
                             f"gpu=({vg[z, y, x]},{wg[z, y, x]}) oracle=({vo[z, y, x]},{wo[z, y, x]})")
    assert sg == so, (label, sg, so)


def workload_steps(w, n_scans=None):
    """Scan/shift steps of a synthetic workload: shift whenever the planned origin changes."""
    steps = []
    cur = tuple(w.params["origin"])
    n = len(w.scans) if n_scans is None else n_scans
    for i in range(n):
        if tuple(w.origins[i]) != cur:
            cur = tuple(w.origins[i])
            steps.append(("shift", cur))
        steps.append(("scan", w.scans[i], w.poses[i]))
    return steps
