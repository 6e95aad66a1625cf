"""Multi-GPU path of the benchmark on the CPU: replicas of the evaluation
(each rank its own users' windows, no data-path exchange) aggregated with a
gloo barrier, a sum of windows and a max of times, world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    r, w, local = bench.dist_setup()
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    # rank 0 processed 32 windows in 2 s, rank 1 processed 32 windows in 4 s
    v = bench.job_throughput(w, 32, 2.0 if rank == 0 else 4.0)
    out[rank] = v
    import torch.distributed as dist
    dist.destroy_process_group()


def test_replica_throughput_over_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0] == out[1] == pytest.approx(64 / 4.0)
