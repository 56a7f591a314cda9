"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own replica;
the job time is the slowest rank's and the throughput counts both replicas.
(Every GPU run of this project has one GPU, so the multi-GPU path is replicas
only; this covers its host-side logic.)"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, l = bench.dist_env()
    assert (r, w, l) == (rank, world, rank)
    t_local = 0.010 * (rank + 1)          # rank 1 is the slow one
    t = bench.max_over_ranks(t_local, world)
    v = bench.job_throughput(1000, world, t)
    out[rank] = (t, v)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        t, v = out[rank]
        assert t == pytest.approx(0.020)
        assert v == pytest.approx(2 * 1000 / 0.020)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
    assert bench.job_throughput(10, 1, 0.5) == 20.0


def test_reference_arm_prints_on_rank_zero_only(repo_root):
    """Under torchrun the reference arm (the oracle on the host) runs on rank 0
    alone; the other ranks exit 0 without work or output."""
    import subprocess
    import sys
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(repo_root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
