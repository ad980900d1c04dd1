"""Multi-GPU replicas, host side (gloo, world size 2, CPU): the whole-job time is
the maximum over ranks, the whole-job throughput counts every rank's pixels, and
only rank 0 prints the reference arm's line."""
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


def _worker(rank, world, port, times, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)

    def reduce_max(v):
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    t, gpix = bench.aggregate(times[rank], world, reduce_max)
    out[rank] = (t, gpix)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_pixels():
    import bench
    port = _free_port()
    times = [0.25, 0.40]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, times, out), nprocs=2, join=True)
    for r in range(2):
        t, gpix = out[r]
        assert t == 0.40
        assert gpix == pytest.approx(2 * 4 * bench.NPIX / (0.40e-3) / 1e9)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
