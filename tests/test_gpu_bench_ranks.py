"""bench.py under torchrun with two ranks on one GPU: the sharded headline
integral (a range of sample indices per rank, one all-reduce per iteration),
max-over-ranks timing and rank 0's JSON line.  The ranks exchange through the
gloo backend on the host, so no kernel of one rank waits on the other."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_shard_the_headline_integral():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--gpus", "2", "--steps", "2", "--warmup", "3",
           "--legs", "e2e", "--no-cpu-baseline"]
    env = dict(os.environ, VEGAS_BENCH_DIST_BACKEND="gloo")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["n_gpus"] == 2 and line["scaling"] == "weak" and line["steps"] == 2
    assert line["value"] > 0 and line["e2e"]["value"] > 0
    # 27 launches per step, one sum-installing launch per adapting iteration
    # (10), one for the five fixed-grid rows together and one grid digest per
    # step for the ranks' comparison
    assert line["gpu_launches"] == (27 + 10 + 1 + 1) * 2
    res = line["result"]["fp32"]
    assert abs(res["mean"] - line["result"]["exact"]) < 6 * res["sigma"]
