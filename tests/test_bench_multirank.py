"""The multi-GPU form of the benchmark is replicas only: each rank renders its
own frames and the job's frames/s is (ranks x frames) / slowest rank's time.
Checked on CPU with two gloo ranks: the aggregation takes the maximum time
over ranks, and the reference arm prints from rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (r + 1) * 100 ms for the first arm, 50 ms for the second
    ms, fps = bench.aggregate_ranks([(rank + 1) * 100.0, 50.0], steps=20, world=world, dist=dist, device="cpu")
    q.put((rank, ms, fps))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_is_max_over_ranks_and_counts_all_frames():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, ms, fps in out:
        assert ms == [200.0, 50.0]
        assert fps == [2 * 20 / 0.2, 2 * 20 / 0.05]


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config", "tiny",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
