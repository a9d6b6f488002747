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


def test_flat_gradient_views_are_aligned_and_disjoint():
    """The pipeline's gradient buffers are views of one allocation: each
    starts on a 256-byte boundary, none overlaps another, and one fill
    zeroes them all."""
    import torch
    from paper_2509_17083_gb300.pipeline import _FlatGrads
    shapes = [(7, 3), (5,), (16, 2048, 2), (64, 32), (3, 64), (1,), (0, 2)]
    f = _FlatGrads(shapes, "cpu")
    spans = []
    for v, sh in zip(f.views, shapes):
        assert tuple(v.shape) == sh
        assert v.untyped_storage().data_ptr() == f.buf.untyped_storage().data_ptr()
        # the offset within the allocation (a zero-element view may report a
        # null data pointer, so the storage offset is the measure)
        off = v.storage_offset() * 4
        assert off % 256 == 0
        spans.append((off, off + v.numel() * 4))
        v.fill_(1.0)
    spans.sort()
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    assert sum(v.numel() for v in f.views) == int(f.buf.sum().item())
    f.zero_()
    assert not any(v.any() for v in f.views)
    assert f.owns(f.views[0]) and not f.owns(torch.zeros(3))
