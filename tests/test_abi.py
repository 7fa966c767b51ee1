"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports every
symbol include/*.h declares, validates arguments on the host, and is
independent of the oracle (no shared symbols, no imports either way)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(tsdf_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def cuda_lib():
    from paper_2310_05766_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("tsdf_map_create", "tsdf_map_destroy", "tsdf_integrate", "tsdf_shift", "tsdf_read",
                     "tsdf_stats", "tsdf_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol(cuda_lib):
    missing = [n for n in _declared_functions() if not hasattr(cuda_lib, n)]
    assert not missing, missing


def test_library_is_sm103a_and_oracle_free(cuda_lib):
    from paper_2310_05766_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    assert "orc_" not in out
    # the oracle library exports nothing of the CUDA library either
    import oracle
    out2 = subprocess.run(["nm", "-D", "--defined-only", oracle.build()], capture_output=True, text=True).stdout
    assert "tsdf_" not in out2
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_no_cross_imports():
    pkg = os.path.join(ROOT, "paper_2310_05766_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            txt = open(f).read()
            assert not re.search(r"^\s*(import|from)\s+oracle", txt, flags=re.M), f
            assert "tsdf_oracle" not in txt, f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".py", ".cpp")):
            txt = open(f).read()
            assert "paper_2310_05766_gb300" not in txt, f
            assert "tsdf.h" not in txt, f


def test_host_side_validation_without_gpu():
    from paper_2310_05766_gb300 import binding as b
    base = dict(dims=(64, 64, 64), voxel_size=0.05, tau=0.2, w_max=64, delta_z=0.01, r_min=0.3, r_max=20.0,
                reduce=0, origin=(-32, -32, -32))
    bad = [dict(base, dims=(60, 64, 64)), dict(base, dims=(4, 64, 64)), dict(base, tau=0.01),
           dict(base, w_max=0), dict(base, w_max=40000), dict(base, delta_z=-1.0), dict(base, delta_z=float("nan")),
           dict(base, r_max=0.1), dict(base, reduce=2), dict(base, origin=(-31, -32, -32)),
           dict(base, voxel_size=0.0), dict(base, dims=(32768, 32768, 8)),
           dict(base, origin=((1 << 23) + 8, 0, 0)), dict(base, origin=(0, 0, -(1 << 23) - 8)),
           dict(base, flags=4), dict(base, flags=-1)]
    for p in bad:
        h = ctypes.c_void_p()
        rc = b.lib().tsdf_map_create(ctypes.byref(b.make_params(p)), ctypes.byref(h))
        assert rc == b.TSDF_ERR_INVALID, p
        assert h.value is None
    assert b.lib().tsdf_map_create(None, None) == b.TSDF_ERR_INVALID
    assert b.tsdf_error_string(b.TSDF_ERR_TIMEOUT) == "device wait timed out"
    assert b.tsdf_error_string(12345) == "unknown error"
    pose = (ctypes.c_float * 12)()
    assert b.lib().tsdf_integrate(None, None, 0, pose, None) == b.TSDF_ERR_INVALID
    assert b.lib().tsdf_shift(None, None, None) == b.TSDF_ERR_INVALID
    assert b.lib().tsdf_map_set_store_file(None, b"store.bin", 0) == b.TSDF_ERR_INVALID


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2310_05766_gb300 import binding as b, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "nope.so"))
    monkeypatch.setattr(b, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        b.lib()


def test_binding_constants_match_the_header():
    """Every integer #define of include/tsdf.h that the Python binding also
    defines has the same value there, and the binding defines all error codes,
    options and mode constants."""
    from paper_2310_05766_gb300 import binding as b
    text = open(os.path.join(ROOT, "include", "tsdf.h")).read()
    consts = {}
    for m in re.finditer(r"^#define\s+(TSDF_\w+)\s+([-+()<\d\sL]+?)\s*(?:/\*.*)?$", text, flags=re.M):
        expr = m.group(2).replace("LL", "")
        consts[m.group(1)] = int(eval(expr, {"__builtins__": {}}))
    assert len(consts) > 30
    assert consts["TSDF_MAX_POINTS"] == (1 << 22) - 1
    required = [n for n in consts if n.startswith(("TSDF_ERR_", "TSDF_OPT_", "TSDF_REDUCE_", "TSDF_REDUCTION_",
                                                  "TSDF_FLAG_", "TSDF_BATCH_OPT_"))] + ["TSDF_OK"]
    missing = [n for n in required if not hasattr(b, n)]
    assert not missing, missing
    wrong = [(n, v, getattr(b, n)) for n, v in consts.items() if hasattr(b, n) and getattr(b, n) != v]
    assert not wrong, wrong
