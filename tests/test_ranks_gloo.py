"""The multi-GPU path of bench.py is replicas only: every rank renders its own
copy of the frame and the line aggregates with a barrier, the maximum time
over ranks and the sum of triangles.  These tests run that rank logic as two
gloo processes on the CPU, and the reference arm under torchrun, where rank
0 alone prints."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(world)
    try:
        r.barrier()
        # per-rank frame times and triangle counts: the line takes the slowest
        # rank's time and the triangles of all ranks
        t = r.max(10.0 + rank)
        n = r.sum(1000.0 * (rank + 1))
        q.put((rank, t, n))
    finally:
        r.close()


def test_replica_reductions_over_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(k, world, port, q)) for k in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, t, n in got:
        assert t == 10.0 + world - 1
        assert n == 1000.0 * world * (world + 1) / 2


def test_reference_arm_prints_once_under_torchrun():
    """bench.py --impl reference under torchrun with two ranks: rank 0 times
    the oracle and prints one JSON line, rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--tiles", "2", "--cells", "64",
           "--W", "64", "--H", "36"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
