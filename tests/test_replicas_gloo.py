"""The multi-GPU path of the bench is replicas only: each rank times its own evaluations, the job
time is the maximum over ranks and the rate counts every rank's evaluations.  Checked with two
gloo ranks on CPU."""
import os
import socket
import sys

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_max, rate = bench.aggregate(100.0 * (rank + 1), 3, dist, "cpu")
    out[rank] = (ms_max, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_time_and_job_rate():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        ms_max, rate = out[r]
        assert ms_max == 200.0
        assert abs(rate - 2 * 3 / 0.2) < 1e-9


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench
    ms_max, rate = bench.aggregate(250.0, 5)
    assert ms_max == 250.0 and abs(rate - 20.0) < 1e-12
