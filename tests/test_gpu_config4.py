"""Multi-view training step as one CUDA graph: 3M Gaussians in a radius-2
ball, 8 cameras on a ring (1297x840), 16-level 2^21 BF16 grids.

Every call of the C ABI is asynchronous on the caller's stream with no host
read inside, so the whole 8-view step (forward, loss, reverse of every
stage) is captured once and replayed. The replay must reproduce the eager
step: images and integer outputs exactly, gradients up to the order of
float atomics. The views share one scratch; saving the gathered features
per view (the default) against gathering them again in the reverse
(recompute, features only in the shared scratch) trades memory for time;
both give the same gradients.
"""
import numpy as np
import pytest
import torch

from paper_2509_17083_gb300 import hyrf as H
from paper_2509_17083_gb300 import synth
from paper_2509_17083_gb300.pipeline import DeviceModel, ViewRenderer, shared_workspaces
from tests.gpu_util import cuda_f32, np_, rel_l2

pytestmark = pytest.mark.gpu

# Float atomics add in a different order on every run: a coarse-level table
# entry sums ~1e6 contributions of both signs per step (8 views x 1M+
# Gaussians), whose order-dependent rounding (~sqrt(1e6) x 2^-24 of the
# partial sums) reaches ~1e-4 of the entry. Images and integers are exact.
ORDER_TOL = 5e-4


def _setup(save_features, n=3_000_000):
    w = synth.config4(n=n)
    m = DeviceModel(w)
    views = []
    ws = shared_workspaces()  # the views run one after the other: one scratch
    for cam, tgt in zip(w.cams, w.targets):
        r = ViewRenderer(m, cam, w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale,
                         save_features=save_features, workspaces=ws)
        t = cuda_f32(tgt)
        r.fit_capacity(t)
        views.append((r, t))
    return w, m, views


def _step(m, views):
    m.zero_grad()
    for r, t in views:
        r.step(t)


def _grads(m):
    out = {}
    for k, v in m.grad.items():
        for j, x in enumerate(v if isinstance(v, list) else [v]):
            out[f"{k}{j}"] = np_(x).copy()
    return out


def test_eight_view_step_replays_as_one_cuda_graph():
    w, m, views = _setup(True)
    for r, _ in views:
        r.status.zero_()
    _step(m, views)  # eager reference (also warms every workspace)
    torch.cuda.synchronize()
    for r, _ in views:
        assert H.read_status(r.status) == 0
    ref_img = [np_(r.C).copy() for r, _ in views]
    ref_inst = [int(r.n_inst.item()) for r, _ in views]
    ref = _grads(m)
    launches0 = H.launch_count()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            _step(m, views)
    torch.cuda.current_stream().wait_stream(s)
    captured = H.launch_count() - launches0
    assert captured > 8 * 30  # every stage of every view went into the graph
    for _ in range(2):
        for r, _ in views:
            r.C.zero_()
        g.replay()
    torch.cuda.synchronize()
    for (r, _), img, k in zip(views, ref_img, ref_inst):
        assert H.read_status(r.status) == 0
        assert int(r.n_inst.item()) == k
        assert np.array_equal(np_(r.C), img)
    got = _grads(m)
    for k, v in ref.items():
        assert rel_l2(got[k], v) < ORDER_TOL, k
    # timing: graph replay against eager issue of the same work
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    for _ in range(3):
        g.replay()
    ev[1].record()
    ev[2].record()
    for _ in range(3):
        _step(m, views)
    ev[3].record()
    torch.cuda.synchronize()
    graph_ms, eager_ms = ev[0].elapsed_time(ev[1]) / 3, ev[2].elapsed_time(ev[3]) / 3
    print(f"8-view step: graph {graph_ms:.2f} ms, eager {eager_ms:.2f} ms, {captured} launches")
    assert graph_ms < eager_ms * 1.05


def test_saved_features_against_recompute_memory_and_gradients():
    res = {}
    for save in (True, False):
        torch.cuda.empty_cache()
        torch.cuda.reset_peak_memory_stats()
        w, m, views = _setup(save, n=1_000_000)
        _step(m, views)
        torch.cuda.synchronize()
        res[save] = (torch.cuda.max_memory_allocated(), _grads(m))
        del w, m, views
    peak_save, g_save = res[True]
    peak_re, g_re = res[False]
    print(f"peak memory 8 views x 1M Gaussians: saved features {peak_save / 2**30:.2f} GiB, "
          f"recompute {peak_re / 2**30:.2f} GiB")
    assert peak_re < peak_save
    for k, v in g_save.items():
        assert rel_l2(g_re[k], v) < ORDER_TOL, k


def test_recompute_views_capture_as_one_cuda_graph():
    """Without saved features the views use no second stream; the step still
    captures (a join on an idle stream would break the capture)."""
    w, m, views = _setup(False, n=200_000)
    _step(m, views)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            _step(m, views)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    for r, _ in views:
        assert H.read_status(r.status) == 0
