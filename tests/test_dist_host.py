"""bench.py's multi-rank path on CPU with the gloo backend and two ranks launched by torch.distributed.run: the
reductions behind `value` (slowest rank's time, all ranks' pairs), one independent facade component per rank, and
the reference arm's rule that rank 0 alone runs and prints while the other ranks exit 0."""
import json
import os
import re
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout=600):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2", "--master-addr",
           "127.0.0.1", "--master-port", str(_port()), *args]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)


def test_reductions_and_components_two_ranks():
    p = _torchrun([os.path.join("tests", "dist_worker.py")])
    assert p.returncode == 0, p.stderr[-2000:]
    rows = {int(m.group(1)): json.loads(m.group(2)) for m in re.finditer(r"RANK(\d+) (\{[^\n]*?\})(?=RANK|\n|$)",
                                                                          p.stdout)}
    assert sorted(rows) == [0, 1]
    import scenes
    for r, d in rows.items():
        assert d["world"] == 2 and d["max"] == 2.5 and d["sum"] == 300.0
        assert d["signatures"] == rows[0]["signatures"]   # every rank saw the same gathered list
    assert rows[0]["seed"] == scenes.SEED_BASE + 2           # rank 0 matches the standard facade
    assert rows[1]["seed"] != rows[0]["seed"]
    assert rows[0]["signatures"][0] != rows[0]["signatures"][1]   # the two components differ


def test_reference_arm_two_ranks():
    p = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"])
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1                                    # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
