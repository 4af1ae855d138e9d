"""The multi-rank path of bench.py on CPU (world size 2, gloo): replicas
meet at the barrier, the timing taken is the slowest rank's, and only rank 0
runs and reports the reference arm (the other ranks return nothing)."""
import argparse
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        bench.barrier(world)
        slowest = bench.max_over_ranks(1.5 + rank, world)
        bench.SWEEP = [(2, 2), (3, 2)]
        bench.CPU_SAMPLE_N = 2
        line = bench.reference_arm(argparse.Namespace(steps=1, warmup=1), rank, world)
        results[rank] = (slowest, line is not None, line["n_gpus"] if line else None)
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_replica_ranks_gloo():
    world = 2
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), results), nprocs=world, join=True)
        got = dict(results)
    assert got[0][0] == got[1][0] == 2.5          # max over the ranks' times
    assert got[0][1] and got[0][2] == world       # rank 0 reports the reference line
    assert not got[1][1]                          # rank 1 reports nothing
