"""The multi-process host path of bench.py on CPU (gloo, world size 2).

The scoring path does not shard (one GPU per replica), so a multi-GPU run is
N independent replicas: a barrier around the timed region, the maximum of
the ranks' times, the sum of their work, and rank 0 alone printing one JSON
line.  These tests run that host logic with two gloo processes.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    w, r, local = bench.dist_env()
    dist = bench.dist_init(w)
    bench.barrier(dist)
    mx = bench.max_over_ranks(dist, 1.5 + r)
    sm = bench.sum_over_ranks(dist, float(r + 1))
    bench.barrier(dist)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "max": mx, "sum": sm}, f)
    dist.destroy_process_group()


def test_rank_reductions_over_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, g in enumerate(got):
        assert g == {"world": 2, "rank": r, "max": 2.5, "sum": 3.0}


def test_reference_arm_under_torchrun_prints_once():
    """Two ranks: rank 0 times the oracle and prints the line, rank 1 exits
    without work; both exit 0."""
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
