"""bench.py --gpus N without an outside launcher: the script re-runs itself as
N ranks under torch.distributed.run (one process per GPU). Driven here end to
end on the CPU through the reference arm (the oracle on the host cores), where
rank 0 alone works and prints the line and every other rank exits 0."""
import json
import os
import subprocess
import sys

import pytest

pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpus_2_spawns_two_ranks_and_rank0_prints_one_line():
    env = {k: v for k, v in os.environ.items()
           if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3", "--ref-budget", "1"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["steps"] == 1 and out["warmup"] == 3
    assert out["value"] > 0 and out["cpu_baseline"]["kind"] == "oracle"
