"""The multi-rank harness of bench.py on the host, launched the way the
benchmark is for N > 1 (torch.distributed.run, one process per rank,
rendezvous on 127.0.0.1): gloo ranks agree on the slowest rank's time, and the
reference arm prints one JSON line from rank 0 while the other rank exits 0
without output.  The data path itself needs a GPU and replicates per rank (no
data-path collective)."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout=300):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    env = dict(os.environ, OMP_NUM_THREADS=os.environ.get("OMP_NUM_THREADS", "4"))
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)


def _json_lines(text):
    return [json.loads(l) for l in text.splitlines() if l.startswith("{")]


def test_max_over_ranks_two_gloo_ranks(tmp_path):
    r = _torchrun([os.path.join("tests", "_gloo_max.py"), str(tmp_path)])
    assert r.returncode == 0, r.stderr[-2000:]
    got = [json.load(open(tmp_path / ("rank%d.json" % k))) for k in range(2)]
    assert [d["rank"] for d in got] == [0, 1] and all(d["world"] == 2 for d in got)
    assert all(d["max"] == 3.5 for d in got)          # 1.5 on rank 0, 3.5 on rank 1


def test_reference_arm_two_ranks_prints_once():
    r = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--workload", "small_2d",
                   "--steps", "1", "--warmup", "1", "--cpu-seconds", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
