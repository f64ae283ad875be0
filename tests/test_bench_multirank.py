"""bench.py's multi-rank plumbing on the CPU (gloo, world size 2).

Under torchrun each rank drains its own replica of the workload; `value` is
all ranks' messages divided by the slowest rank's time (weak scaling).  This
checks the reductions that compute it, and the reference arm's rule that
only rank 0 runs and prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, outdir: str) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    r, _, w = bench.dist_env()
    bench.dist_init(w, "gloo")
    # rank r drained 1000 (r + 1) messages in 0.5 (r + 1) seconds
    msgs = bench.allreduce_sum(1000.0 * (r + 1), w)
    secs = bench.allreduce_max(0.5 * (r + 1), w)
    bench.barrier(w)
    with open(os.path.join(outdir, f"rank{r}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "msgs": msgs, "secs": secs, "value": msgs / secs}, f)
    dist.destroy_process_group()


def test_reductions_give_whole_job_rate(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    rows = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for row in rows:
        assert row["world"] == 2
        assert row["msgs"] == 3000.0          # sum over ranks
        assert row["secs"] == 1.0             # the slowest rank
        assert row["value"] == 3000.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--cpu-seconds", "1", "--gpus", "2"]
    r1 = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    env.update(RANK="0", LOCAL_RANK="0")
    r0 = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=120, cwd=ROOT)
    assert r0.returncode == 0, r0.stderr
    lines = [ln for ln in r0.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
