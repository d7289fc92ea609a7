"""Rank logic of bench.py under torchrun, on CPU with gloo (world size 2):
max-over-ranks timing, the whole-job rate, and the reference arm's
"rank 0 alone" rule."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_rank_max_and_rate(tmp_path):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "tests", "multirank_worker.py"), str(tmp_path)]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    recs = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert sorted(r["rank"] for r in recs) == [0, 1]
    for r in recs:
        assert r["world"] == 2
        assert r["worst"] == 150.0
        # 1000 nodes per rank x 2 ranks x 5 stages x 3 steps over 0.15 s
        assert abs(r["rate"] - 1000 * 2 * 5 * 3 / 0.15) < 1e-6


def test_reference_arm_nonzero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                         capture_output=True, text=True, timeout=120, env=env, cwd=ROOT)
    assert out.returncode == 0
    assert out.stdout.strip() == ""
