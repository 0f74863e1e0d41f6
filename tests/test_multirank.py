"""The N>1 bench path on CPU with two gloo ranks: every rank marches its own
batch of plane waves (independent problems, no data-path collective); the job
throughput uses the slowest rank's time."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2510_07989_gb300.inputs import meshes as MS
    vals = bench.reduce_max([10.0 + rank, 100.0 - rank], world)
    exc = MS.fibonacci_batch(4, 0.1, seed=20251007 + rank)
    out[rank] = (vals, exc.p.copy(), bench.throughput(world, 4, 10, vals[0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_and_distinct_batches():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    v0, p0, thr0 = out[0]
    v1, p1, thr1 = out[1]
    assert v0 == v1 == [11.0, 100.0]            # max over ranks of both timings
    assert thr0 == thr1 == pytest.approx(2 * 4 * 10 / 0.011)
    assert not np.allclose(p0, p1)               # each rank has its own plane waves


def test_reference_arm_under_torchrun_two_ranks():
    """The driver's N > 1 reference invocation: under torchrun with two ranks
    only rank 0 runs the oracle and prints; the other rank exits 0 without
    work, so the job prints exactly one JSON line (small torus, one step)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(root, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--workload", "torus32x12", "--steps", "1", "--warmup", "0"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
