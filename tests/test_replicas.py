"""Multi-GPU runs are independent replicas (one view per rank, no
collective in the data path): the benchmark's only cross-rank step is the
maximum of the step time. Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        out[rank] = bench.replica_max(1.5 + rank)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_step():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn", join=True)
    assert dict(out) == {0: 2.5, 1: 2.5}
    assert bench.whole_job_rate(2.5, ws) == pytest.approx(800.0)
