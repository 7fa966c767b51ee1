"""Host logic: the global store's chunk index (a C++ header of the library),
compiled with the host compiler and checked against std::map."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2310_05766_gb300", "csrc")


def test_chunk_index_matches_std_map(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "chunk_index_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "chunk_index_check.cpp"), "-o", exe],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr


def test_chunk_store_slots_across_tiers(tmp_path):
    """The store's slot bookkeeping (csrc/chunk_store.h) over 4000 random shifts
    with a small device tier: stored exactly the chunks that hold data, read
    back as themselves, no shared slots, oldest device chunks moved first."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "chunk_store_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, os.path.join(HERE, "chunk_store_check.cpp"), "-o", exe],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr


def test_chunk_store_file_tier(tmp_path):
    """The store's file tier (csrc/chunk_file.h with csrc/chunk_store.h) over
    3000 random shifts with a real scratch file and the asynchronous writer:
    reads right after writes return the latest content, every re-entering
    chunk reads back the content it left with (from the file or the write
    queue), the host tier stays within its limit, the file is removed when the
    writer is destroyed, and a failed write (past a lowered file size limit)
    is reported by every later call."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "chunk_file_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-pthread", "-I", CSRC, os.path.join(HERE, "chunk_file_check.cpp"),
                    "-o", exe], check=True)
    scratch, scratch2 = str(tmp_path / "scratch.bin"), str(tmp_path / "scratch2.bin")
    r = subprocess.run([exe, scratch, scratch2], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    assert not os.path.exists(scratch) and not os.path.exists(scratch2)
