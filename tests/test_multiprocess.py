"""The N > 1 path of the benchmark on CPU (no GPU): two ranks over gloo.  Multi-GPU here is
replicas only (every pixel is independent, Sec. 4): each rank renders its own frame with its own
seed, the job's time is the maximum over ranks and the job's throughput counts all ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_init()
    bench.barrier(w)
    mx = bench.allreduce_max(float(10 * (r + 1)), w)
    seed = bench.replica_seed(r)
    q.put((r, w, dist.get_backend(), mx, seed))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [x[0] for x in res] == [0, 1] and all(x[1] == world for x in res)
    assert all(x[2] == "gloo" for x in res)
    assert all(x[3] == 20.0 for x in res)                 # max over ranks
    assert len({x[4] for x in res}) == world              # one seed per replica


def test_job_value_counts_all_ranks():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_value(1000, 5, 2000.0, 1) == 2500.0
    assert bench.job_value(1000, 5, 2000.0, 4) == 10000.0


def test_reference_arm_under_torchrun_prints_once():
    """Under torchrun the reference arm runs on rank 0 only and prints one JSON line."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--steps", "1", "--warmup", "0", "--workload", "band"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
