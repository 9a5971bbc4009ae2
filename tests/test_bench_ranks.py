"""bench.py's multi-rank timing (replicas, one rank per GPU): the job time is the
slowest rank's, taken with one MAX all-reduce.  Checked with two gloo ranks on
the CPU (the GPU run uses NCCL on the same code path)."""
import os
import socket
import sys
import tempfile

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    got = bench.max_over_ranks(10.0 + 7.5 * rank, dist, "cpu")
    np.save(path + f".{rank}.npy", np.array([got]))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_processes():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "r")
        mp.start_processes(_rank, args=(2, port, path), nprocs=2, start_method="spawn")
        vals = [float(np.load(path + f".{r}.npy")[0]) for r in range(2)]
    assert vals == [17.5, 17.5]


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
