"""The N > 1 path of bench.py on CPU, world size 2 over gloo.

The method needs no data exchange on one GPU (replicas only): a multi-GPU
run is N independent replicas that meet at a barrier around the timed
region, and the job's time is the slowest rank's.  These tests run that
host logic in two processes: the max-over-ranks reduction and barrier,
and the reference arm under torchrun (rank 0 alone runs and prints one
JSON line, the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    class Args:
        pass
    got_world, got_rank, _ = bench.dist_setup(Args())
    bench.barrier(got_world)
    slowest = bench.max_over_ranks(got_world, 10.0 + 5.0 * rank)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"world": got_world, "rank": got_rank, "max": slowest}, fh)
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_gloo(tmp_path):
    port = free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    recs = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert [r["rank"] for r in recs] == [0, 1]
    assert all(r["world"] == 2 for r in recs)
    assert all(r["max"] == 15.0 for r in recs)  # every rank sees the slowest rank's time


@pytest.mark.slow
def test_reference_arm_under_torchrun():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2
    assert rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0
