"""The multi-GPU bench path on CPU (gloo, world size 2): every rank runs its own replica, the job's
time is the slowest replica's (max over ranks), and the reference arm runs on rank 0 only."""
import io
import os
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + rank * 0.5, dist, "cpu")       # replica times 1.0 and 1.5
    buf = io.StringIO()
    if rank != 0:
        # the reference arm does no work and prints nothing on ranks other than 0
        class A:
            cpu_sample_evals, warmup, steps, gpus = 1, 0, 1, world
        with redirect_stdout(buf):
            bench.run_reference(A(), rank, world)
    out[rank] = (t, buf.getvalue())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = 29500 + (os.getpid() % 1000)
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert out[0][0] == 1.5 and out[1][0] == 1.5
    assert out[1][1] == ""
