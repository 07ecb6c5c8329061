"""The multi-rank (replicas) path of bench.py on CPU: two gloo ranks run the
reference arm; only rank 0 prints one JSON line; the other exits 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_two_gloo_ranks_print_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29531", "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


WORKER = r'''
import os, sys, json
sys.path.insert(0, os.environ["MRS_ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
# each rank's own elapsed time; the bench reports the slowest rank's
t = bench.max_over_ranks(10.0 + 5.0 * rank, world)
one = bench.max_over_ranks(3.0, 1)
with open(os.path.join(os.environ["MRS_OUT"], "rank%d.json" % rank), "w") as f:
    json.dump({"rank": rank, "max": t, "single": one}, f)
dist.destroy_process_group()
'''


def test_max_over_ranks_on_two_gloo_ranks(tmp_path):
    # the GPU arm's cross-rank timing reduction, exercised on CPU ranks
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29533", str(script)]
    env = dict(os.environ, MRS_ROOT=ROOT, MRS_OUT=str(tmp_path), OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    got = [json.loads((tmp_path / f"rank{k}.json").read_text()) for k in (0, 1)]
    assert sorted(g["rank"] for g in got) == [0, 1]
    assert all(g["max"] == 15.0 and g["single"] == 3.0 for g in got)
