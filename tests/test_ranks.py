"""The N > 1 benchmark path, on CPU with the gloo backend (world size 2).

Each rank runs its own replica; the only cross-rank steps are a barrier and
the max over ranks of the timed region.  The reference arm runs on rank 0
only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [3.0, 5.0][rank]
    t, v = bench.aggregate(local_ms, 100, 4, world, dist, "cpu")
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_two_rank_aggregation_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, v in out:
        assert t == 5.0                                 # slowest rank
        assert v == pytest.approx(2 * 100 * 4 / 5e-3)   # all ranks' units over that time


def test_single_rank_aggregation_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    t, v = bench.aggregate(2.0, 10, 3, 1)
    assert t == 2.0 and v == pytest.approx(10 * 3 / 2e-3)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
