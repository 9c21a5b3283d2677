"""The multi-rank path of bench.py (independent replicas, one per GPU) on
CPU: two gloo ranks, the whole-job time is the slowest rank's and the work is
the sum over ranks; the reference leg prints only on rank 0."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u = bench.aggregate(dist, 1.0 + rank, 100.0 * (rank + 1))
    q.put((rank, t, u))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u in res:
        assert t == 2.0          # max over ranks
        assert u == 300.0        # sum over ranks


def test_single_process_aggregation_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.aggregate(None, 0.5, 42.0) == (0.5, 42.0)


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_leg_prints_once_under_torchrun():
    """bench.py --impl reference launched as 2 ranks: rank 0 alone runs the
    oracle and prints one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--grid", "64", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    for k in ("metric", "unit", "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert k in d
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
