"""The N > 1 host logic of bench.py on CPU: gloo, world size 2.

Masks are independent, so N ranks run N replicas; the only collectives are
the timing barrier and the max over ranks. Here: the max-over-ranks reduction
under gloo, and the reference arm launched through torchrun, where rank 0
alone prints one JSON line and every rank exits 0.
"""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
rank, ws = bench.dist_setup("gloo")
assert ws == 2
bench.barrier(ws)
m = bench.max_over_ranks(float(rank + 1) * 1.5, ws)
assert m == 3.0, m
total = bench.max_over_ranks(10.0 * (rank + 1), ws) / (4 * ws)
assert abs(total - 2.5) < 1e-12
print("rank", rank, "ok")
dist.destroy_process_group()
"""


def run_torchrun(args, timeout=300):
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port)] + args
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="2")
    return subprocess.run(cmd, capture_output=True, text=True, timeout=timeout, cwd=ROOT, env=env)


def test_max_over_ranks_gloo(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER.format(root=ROOT))
    r = run_torchrun([str(script)])
    assert r.returncode == 0, r.stderr[-3000:]
    assert r.stdout.count("ok") == 2


@pytest.mark.slow
def test_reference_arm_under_torchrun():
    r = run_torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
                      "--ref-sample-iters", "1"], timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "ms/mask" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
