"""The replica path of bench.py on CPU with gloo, world size 2: the job time
is the slowest rank's and the work is the sum over ranks."""
from __future__ import annotations

import os

import torch.multiprocessing as mp


def _rank(rank, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    ms, units = bench.aggregate_replicas(10.0 + 5.0 * rank, 1000 * (rank + 1), 2)
    out[rank] = (ms, units)
    dist.destroy_process_group()


def test_replica_aggregation_gloo():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (15.0, 3000.0)


def test_single_process_is_identity():
    import bench
    assert bench.aggregate_replicas(7.5, 123, 1) == (7.5, 123)
