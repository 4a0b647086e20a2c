"""Replicated runs (one process per GPU, no data-path collective): the
bench's whole-job aggregation over world_size 2, on CPU with gloo."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), RW_BACKEND="gloo")
    import bench
    got_ws, got_rank, got_local = bench._dist()
    units, ms = bench.aggregate(100.0 * (rank + 1), 10.0 * (rank + 1), got_ws)
    out[rank] = (got_ws, got_rank, got_local, units, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ws = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(ws, port, out), nprocs=ws, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(ws):
        got_ws, got_rank, got_local, units, ms = res[rank]
        assert (got_ws, got_rank, got_local) == (2, rank, rank)
        # every rank sees the job total (100 + 200 units) and the slowest rank's 20 ms
        assert units == 300.0 and ms == 20.0


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(123.0, 4.5, 1) == (123.0, 4.5)
