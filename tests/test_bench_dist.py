"""bench.py's multi-rank bookkeeping on CPU ranks (gloo, world size 2): the
max-over-ranks timing reduction and barrier, and the reference arm printing
one line from rank 0 while the other rank exits without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def torchrun(args, timeout=300):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % free_port(), *args]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


def test_max_over_ranks_and_barrier(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(
        "import sys\n"
        "import bench\n"
        "ws, rank, local = bench.dist_setup()\n"
        "v = bench.max_over_ranks(10.0 * (rank + 1), ws)\n"
        "bench.barrier(ws)\n"
        "open(sys.argv[1] + '/rank%d.txt' % rank, 'w').write('%d %d %s' % (rank, ws, v))\n")
    r = torchrun([str(script), str(tmp_path)])
    assert r.returncode == 0, r.stderr[-2000:]
    got = sorted((tmp_path / ("rank%d.txt" % i)).read_text() for i in range(2))
    assert got == ["0 2 20.0", "1 2 20.0"]


def test_reference_arm_prints_once():
    r = torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                  "--warmup", "0", "--points", "16384"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["unit"] == "ms"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["n"] == 16384 and d["dtype"] == "f64"
