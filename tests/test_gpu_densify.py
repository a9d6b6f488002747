"""Adaptive density control on the GPU against the oracle: gradient
statistics and decisions bit for bit, the rewritten arrays (copies exact,
split positions to float rounding), and a training run that densifies,
prunes and resets opacity while it converges."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2509_17083_gb300 import hyrf as H
from paper_2509_17083_gb300 import synth
from tests.gpu_util import cuda_f32, cuda_i32, np_

pytestmark = pytest.mark.gpu


def _inputs(seed=61, n=100_000, nv=60_000):
    rng = np.random.default_rng(seed)
    vis = np.sort(rng.choice(n, nv, replace=False)).astype(np.int32)
    views = []
    for _ in range(3):
        dm = (rng.standard_normal((nv, 2)) * 2e-7 * rng.uniform(0, 3, (nv, 1))).astype(np.float32)
        nt = rng.integers(0, 4, nv).astype(np.int32)
        views.append((dm, nt))
    alpha = rng.uniform(0, 1, nv).astype(np.float32)
    alpha[: nv // 50] = rng.uniform(0, 0.005, nv // 50)
    scale = np.exp(rng.uniform(-6, -2, (nv, 3))).astype(np.float32)
    quat = synth.random_quats(rng, nv)
    noise = rng.standard_normal((n, 2, 3)).astype(np.float32)
    return rng, n, vis, views, alpha, scale, quat, noise


def test_densify_matches_oracle():
    rng, n, vis, views, alpha, scale, quat, noise = _inputs()
    W, Hh = 1237, 822
    dev = "cuda"
    nv = len(vis)
    d_vis, d_nv = cuda_i32(vis), torch.tensor([nv], dtype=torch.int32, device=dev)
    accum = torch.zeros(n, device=dev)
    count = torch.zeros(n, dtype=torch.int32, device=dev)
    ra, rc = np.zeros(n, np.float32), np.zeros(n, np.int32)
    for dm, nt in views:
        H.hyrf_densify_stats(n=n, vis_ids=d_vis, n_vis=d_nv, d_mean2d=cuda_f32(dm), ntiles=cuda_i32(nt),
                             width=W, height=Hh, accum=accum, count=count)
        ra, rc = oracle.densify_stats(n, vis, dm, nt, W, Hh, ra, rc)
    torch.cuda.synchronize()
    assert np.array_equal(np_(accum).view(np.uint32), ra.view(np.uint32))
    assert np.array_equal(np_(count), rc)
    thr, dense, minop = 2e-4, 0.05, 0.005
    action = torch.zeros(n, dtype=torch.uint8, device=dev)
    row = torch.zeros(n, dtype=torch.int32, device=dev)
    offset = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    n_out = torch.zeros(1, dtype=torch.int64, device=dev)
    H.hyrf_densify_plan(n=n, vis_ids=d_vis, n_vis=d_nv, alpha=cuda_f32(alpha), scale=cuda_f32(scale),
                        accum=accum, count=count, grad_threshold=thr, dense_scale=dense, min_opacity=minop,
                        action=action, row=row, offset=offset, n_out=n_out)
    ract, rrow, roff, rtot = oracle.densify_plan(n, vis, alpha, scale, ra, rc, thr, dense, minop)
    torch.cuda.synchronize()
    assert np.array_equal(np_(action), ract)
    assert np.array_equal(np_(row), rrow)
    assert np.array_equal(np_(offset), roff)
    assert int(n_out.item()) == rtot
    counts = np.bincount(ract, minlength=4)
    assert counts[1] > 100 and counts[2] > 100 and counts[3] > 100, counts  # every action occurs
    N2 = rtot
    pos = rng.standard_normal((n, 3)).astype(np.float32)
    se = rng.uniform(-5, -2, n).astype(np.float32)
    col = rng.standard_normal((n, 3)).astype(np.float32)
    mst = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    srcs = [(pos, H.REMAP_POSITION), (se, H.REMAP_SCALE_LOGIT), (col, H.REMAP_PARAM), (mst, H.REMAP_STATE)]
    arrays = []
    for a, kind in srcs:
        src = cuda_f32(a)
        dst = torch.full((N2,) + a.shape[1:], float("nan"), device=dev)
        arrays.append((src, dst, kind))
    H.hyrf_densify_apply(arrays, n=n, action=action, row=row, offset=offset, scale=cuda_f32(scale),
                         quat=cuda_f32(quat), noise=cuda_f32(noise), split_log_scale=math.log(1.6))
    torch.cuda.synchronize()
    for (a, kind), (_, dst, _) in zip(srcs, arrays):
        ref = oracle.densify_apply(ract, rrow, roff, scale.astype(np.float64), quat.astype(np.float64),
                                   noise.astype(np.float64), math.log(1.6), a, kind)
        got = np_(dst).astype(np.float64)
        assert np.isfinite(got).all(), kind
        if kind in (H.REMAP_PARAM, H.REMAP_STATE):
            assert np.array_equal(got, ref), kind
        else:
            np.testing.assert_allclose(got, ref, rtol=1e-6, atol=1e-7)


def test_reset_opacity():
    a = torch.tensor([-1.0, -6.0, 3.0], device="cuda")
    m, v = torch.ones(3, device="cuda"), torch.ones(3, device="cuda")
    H.hyrf_reset_opacity(a, math.log(0.01 / 0.99), m, v)
    torch.cuda.synchronize()
    lim = np.float32(math.log(0.01 / 0.99))
    assert np_(a).tolist() == [lim, -6.0, lim]
    assert np_(m).tolist() == [0.0] * 3 and np_(v).tolist() == [0.0] * 3
