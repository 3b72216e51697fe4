"""Multi-process (world size 2, gloo, CPU) coverage of the replica path of
bench.py: each rank times its own solves; the job value takes the slowest
rank.  The reference arm prints nothing on ranks other than 0."""
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, ms, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = bench.aggregate_ms(ms[rank], world, dist, "cpu")
    q.put((rank, m, bench.solves_per_s(m, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_takes_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ms = [120.0, 150.0]
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, v in res:
        assert m == 150.0
        assert abs(v - 2 * 1000.0 / 150.0) < 1e-12


def test_reference_arm_is_silent_on_nonzero_ranks():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
