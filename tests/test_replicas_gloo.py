"""Multi-GPU layout of the benchmark, exercised on CPU with gloo: every rank
solves an independent replica (its own sources), and the job's numbers are
the slowest rank's time and the sum of the eigenpairs."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, pairs = bench.reduce_job(100.0 + 50.0 * rank, 12.0 + rank, world, "cpu")
    # replicas draw different sources, the same gauge field
    U, src = bench.make_inputs(rank)
    out[rank] = (ms, pairs, float(np.abs(src).sum()), float(np.abs(U).sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_job_aggregation_and_distinct_replicas():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 150.0       # max over ranks
    assert out[0][1] == out[1][1] == 25.0        # sum over ranks
    assert out[0][2] != out[1][2]                # independent sources
    assert out[0][3] == out[1][3]                # shared gauge field


def test_single_rank_is_identity():
    assert bench.reduce_job(3.0, 4.0, 1, "cpu") == (3.0, 4.0)
