"""The N>1 path of bench.py: replicas with no data-path collective; the whole-
job value is world * steps / max-over-ranks time.  Checked with two gloo
ranks on CPU; the reference arm prints only on rank 0."""
import os
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    total = 1.0 + rank            # rank 1 is slower
    v = bench.whole_job_value(total, steps=10, world=world, dist=dist, device="cpu")
    out[rank] = v
    dist.destroy_process_group()


def test_whole_job_value_uses_max_over_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, 29517, out), nprocs=2, join=True)
    assert abs(out[0] - 2 * 10 / 2.0) < 1e-12
    assert out[0] == out[1]


def test_reference_arm_other_ranks_are_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
