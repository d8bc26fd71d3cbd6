"""The N > 1 path of the benchmark on CPU: world size 2 over gloo.

bench.py runs one independent solve per rank (replicas, no data-path
collective); the only communication is the barrier and the maximum of the
per-rank step times, tested here with the gloo backend. The reference arm must
leave ranks other than 0 without work.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = bench.reduce_max(10.0 + rank * 5.0, dist)
    dist.barrier()
    # the reference arm runs on rank 0 only; other ranks return 0 without work
    os.environ["RANK"] = str(rank)
    if rank != 0:
        class A:  # minimal argument object
            s, warmup, steps = 8, 1, 1
        rc = bench.reference_arm(A())
    else:
        rc = 0
    out[rank] = (ms, rc)
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(worker, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[1][1] == 0


def test_reduce_max_without_dist():
    import bench

    assert bench.reduce_max(3.5, None) == 3.5
