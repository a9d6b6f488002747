"""End-to-end GPU parity: one training iteration of a view (all five stages
forward, Eq. 12 loss, all reverse passes) against the composed FP64 oracle,
at sizes the oracle finishes in seconds (several tiles, ragged image edges).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_17083_gb300 import hyrf as H
from paper_2509_17083_gb300 import synth
from paper_2509_17083_gb300.pipeline import DeviceModel, ViewRenderer
from tests.gpu_util import (TOL_GRAD_F32, TOL_GRAD_F32_TRAINED, TOL_IMG_F32, TOL_IMG_F32_TRAINED,
                            cuda_f32, np_, rel_l2)

pytestmark = pytest.mark.gpu

CASES = {
    # full-size config 1 (4,096 Gaussians, 128x128, 16x16 map, L1), its U(+-1e-4) init
    "config1": lambda: synth.config1(),
    # config 1 with trained-like grids (U(+-0.5))
    "config1_trained": lambda: synth.config1(table_init=0.5),
    # config 2 generator at reduced size (map background, L1 + 0.2 D-SSIM)
    "config2_small": lambda: synth.config2(n=20000, width=203, height=157, log2_T=14,
                                           n_clusters=16),
    "config2_small_trained": lambda: synth.config2(n=20000, width=203, height=157, log2_T=14,
                                                   n_clusters=16, table_init=0.5),
    # config 3 generator at reduced size, FP32 variant (exact background)
    "config3_small_f32": lambda: synth.config3(n=30000, width=301, height=203, log2_T=15,
                                               n_clusters=32, precision="f32"),
    "config3_small_f32_trained": lambda: synth.config3(n=30000, width=301, height=203, log2_T=15,
                                                       n_clusters=32, precision="f32",
                                                       table_init=0.5),
}


def _run(w, mask=None, qmask=None):
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
    tgt = cuda_f32(w.targets[0])
    r.fit_capacity(tgt)
    m.zero_grad()
    r.status.zero_()
    r.forward(tgt)
    if mask is not None:
        r.dC.mul_(cuda_f32(mask)[..., None])
    r.backward_render()
    if qmask is not None:
        q = cuda_f32(qmask)
        nv = len(qmask)
        r.d_alpha[:nv].mul_(q)
        for t in (r.d_scale, r.d_quat, r.d_color):
            t[:nv].mul_(q[:, None])
    r.backward_fields()
    torch.cuda.synchronize()
    return m, r


# ReLU kinks: decoder backward inputs are kept only for Gaussians whose
# hidden pre-activations are not within these relative margins of zero (the
# FP32 geometry decoder at initialisation sees inputs ~1e-4 whose rounding
# moves pre-activations by ~1e-3 of their magnitude).
RELU_MARGIN_F32 = (1e-3, 1e-4)


@pytest.mark.parametrize("case", list(CASES))
def test_view_iteration_matches_oracle(case):
    """One iteration vs the oracle. The loss gradient is restricted (on both
    sides) to the pixels the oracle shows to be decision-safe, and the
    decoder backward to the Gaussians away from ReLU kinks, so that both
    differentiate the same smooth function; the image is compared on the
    safe pixels too."""
    w = CASES[case]()
    fw = oracle.render(w.gaussians, w.fields, w.cams[0], w.bg)
    mask = oracle.decision_safe_mask(fw, w.cams[0])
    assert mask.mean() > 0.9, mask.mean()
    qmask = oracle.relu_safe_mask(w.gaussians, w.fields, w.cams[0], fw["ids"], *RELU_MARGIN_F32)
    assert qmask.mean() > 0.5, qmask.mean()
    m, r = _run(w, mask.astype(np.float32), qmask)
    assert H.read_status(r.status) == 0
    L, fw, grads, inter = oracle.loss_and_grads(w.gaussians, w.fields, w.cams[0], w.bg,
                                                w.targets[0], w.ssim_lambda, dC_mask=mask,
                                                query_mask=qmask)
    nv = int(r.n_vis.item())
    assert nv == len(fw["ids"]) and np.array_equal(np_(r.vis_ids)[:nv], fw["ids"])
    trained = case.endswith("_trained")
    err = np.abs(np_(r.C) - fw["C"]).max(-1)
    tol = TOL_IMG_F32_TRAINED if trained else TOL_IMG_F32
    assert err[mask].max() < tol, err[mask].max()
    assert np.quantile(err, 0.999) < 1e-2
    assert abs(float(r.loss.item()) - L) < (1e-4 if trained else 1e-5)
    gtol = TOL_GRAD_F32_TRAINED if trained else TOL_GRAD_F32
    g = m.grad
    for key in ("pos", "alpha_e", "scale_e", "color_e", "geo_table", "rad_table"):
        e = rel_l2(np_(g[key]), grads[key])
        assert e < gtol, (key, e)
    for key in ("geo_W", "geo_b", "col_W", "col_b"):
        for l in range(len(g[key])):
            e = rel_l2(np_(g[key][l]), grads[key][l])
            assert e < gtol, (key, l, e)


def test_two_iterations_are_identical_in_integers():
    w = CASES["config2_small_trained"]()
    m, r = _run(w)
    k1, v1, rg1 = np_(r.keys).copy(), np_(r.vals).copy(), np_(r.ranges).copy()
    n1 = int(r.n_inst.item())
    r.step(cuda_f32(w.targets[0]))
    torch.cuda.synchronize()
    assert int(r.n_inst.item()) == n1
    assert np.array_equal(np_(r.keys)[:n1], k1[:n1])
    assert np.array_equal(np_(r.vals)[:n1], v1[:n1])
    assert np.array_equal(np_(r.ranges), rg1)


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_step_graph_replays_the_eager_step(precision):
    """The training iteration captured as one CUDA graph (StepGraph): a
    replay gives the eager step's image and integers exactly and its
    gradients up to the order of float atomics; a new target written into
    the graph's buffer is used by the next replay."""
    from paper_2509_17083_gb300.pipeline import StepGraph
    w = synth.config3(n=30000, width=301, height=203, log2_T=15, n_clusters=32, precision=precision,
                      table_init=0.3)
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
    tgt = cuda_f32(w.targets[0])
    r.fit_capacity(tgt)
    r.status.zero_()
    m.zero_grad()
    r.forward(tgt, want_keys=False)
    r.backward()
    torch.cuda.synchronize()
    img, nc, loss = np_(r.C).copy(), np_(r.n_contrib).copy(), float(r.loss.item())
    ref = {k: np_(v).copy() for k, v in m.grad.items() if not isinstance(v, list)}
    sg = StepGraph(r, tgt)
    assert sg.launches > 20
    for _ in range(2):
        r.C.zero_()
        sg.replay()
    torch.cuda.synchronize()
    assert H.read_status(r.status) == 0
    assert np.array_equal(np_(r.C), img)
    assert np.array_equal(np_(r.n_contrib), nc)
    # the loss is a sum of per-CTA partial sums added with float atomics
    assert abs(float(r.loss.item()) - loss) <= 1e-5 * abs(loss)
    for k, v in ref.items():
        assert rel_l2(np_(m.grad[k]), v) < 1e-4, k
    # a new target through the graph's buffer
    t2 = torch.rand_like(tgt)
    sg.target.copy_(t2)
    sg.replay()
    torch.cuda.synchronize()
    l2 = float(r.loss.item())
    r.forward(t2, want_keys=False)
    torch.cuda.synchronize()
    assert abs(float(r.loss.item()) - l2) <= 1e-5 * abs(l2)


def test_background_reverse_beside_compositing_reverse():
    """The pipeline's overlapped reverse (background reverse on the second
    stream with d_T_final NULL, compositing reverse from the composited
    image, C - C_fg = T_final c_s) against the sequential one (the
    background's dL/dT_final into the compositing reverse, its table
    scatter forked onto the second stream through scatter_stream)."""
    w = synth.config3(n=30000, width=301, height=203, log2_T=15, n_clusters=32, precision="bf16",
                      table_init=0.3)
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
    assert r._overlap()
    tgt = cuda_f32(w.targets[0])
    r.fit_capacity(tgt)
    r.status.zero_()
    m.zero_grad()
    r.forward(tgt, want_keys=False)
    r.backward()
    torch.cuda.synchronize()
    got = {k: np_(v).copy() for k, v in m.grad.items() if not isinstance(v, list)}
    got["col_W0"] = np_(m.grad["col_W"][0]).copy()
    img = {k: np_(getattr(r, k)).copy() for k in ("d_mean2d", "d_conic", "d_alpha", "d_color")}
    # sequential reference
    m.zero_grad()
    for t in (r.d_mean2d, r.d_conic, r.d_alpha, r.d_color):
        t.zero_()
    g = m.grads_struct()
    H.hyrf_composite_background_backward(r._bg_args(), ws=r.ws["bb"], d_C=r.dC, d_C_fg=None,
                                         d_T_final=r.dT, grads=g, loss_scale=r.loss_scale,
                                         scatter_stream=r.side.cuda_stream)
    H.hyrf_rasterize_backward(r._raster_args(), ws=r.ws["rb"], d_C_fg=r.dC, d_T_final=r.dT,
                              d_mean2d=r.d_mean2d, d_conic=r.d_conic, d_alpha=r.d_alpha, d_color=r.d_color)
    H.hyrf_project_backward(ws=r.ws["p"], n=m.n, pos=m.pos, vis_ids=r.vis_ids, n_vis=r.n_vis, scale=r.scale,
                            quat=r.quat, cam=r.ccam, d_mean2d=r.d_mean2d, d_conic=r.d_conic,
                            d_pos=m.grad["pos"], d_scale=r.d_scale, d_quat=r.d_quat, status=r.status)
    r.backward_fields()
    torch.cuda.current_stream().wait_stream(r.side)
    torch.cuda.synchronize()
    assert H.read_status(r.status) == 0
    for k, v in img.items():
        assert rel_l2(v, np_(getattr(r, k))) < 1e-4, k
    ref = {k: np_(v) for k, v in m.grad.items() if not isinstance(v, list)}
    ref["col_W0"] = np_(m.grad["col_W"][0])
    # the two reverses differ only in the order of the float atomics that
    # sum each table entry's gradient (Eq. 3 reversed): entries summed over
    # thousands of Gaussians with cancelling signs (coarse levels) carry
    # relative differences above 1e-4
    for k, v in ref.items():
        assert rel_l2(got[k], v) < (5e-4 if k.endswith("table") else 1e-4), k
    # a reverse with neither d_T_final nor the image is refused
    with pytest.raises(H.HyrfError):
        H.hyrf_rasterize_backward(r._raster_args(), ws=r.ws["rb"], d_C_fg=r.dC, d_T_final=None,
                                  d_mean2d=r.d_mean2d, d_conic=r.d_conic, d_alpha=r.d_alpha,
                                  d_color=r.d_color)


def test_tile_order_is_a_permutation_and_leaves_the_image_unchanged():
    """hyrf_tile_order: a permutation of the tiles, non-increasing in the bit
    length of each tile's longest pixel list. The compositing forward gives
    the same image, T_final and n_contrib bit for bit in index order, in
    that order and in a random one; an out-of-range entry is reported
    (HYRF_ERR_BOUNDS) and its CTA skipped."""
    w = synth.config3(n=30000, width=301, height=203, log2_T=15, n_clusters=32, precision="bf16",
                      table_init=0.3)
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg)
    r.fit_capacity()
    r.forward(None, want_keys=False)
    torch.cuda.synchronize()
    nt = r.TX * r.TY
    order = np_(r.tile_order).copy()
    assert np.array_equal(np.sort(order), np.arange(nt))
    nc = np_(r.n_contrib)
    pad = np.zeros((r.TY * 16, r.TX * 16), np.int64)
    pad[:nc.shape[0], :nc.shape[1]] = nc
    tmax = pad.reshape(r.TY, 16, r.TX, 16).max(axis=(1, 3)).reshape(-1)
    bits = np.array([int(v).bit_length() for v in tmax])
    assert np.all(np.diff(bits[order]) <= 0)
    ref = [np_(x).copy() for x in (r.C_fg, r.T_final, r.n_contrib)]
    for o in (np.arange(nt), np.random.default_rng(3).permutation(nt)):
        r.tile_order.copy_(torch.as_tensor(o, dtype=torch.int32))
        for x in (r.C_fg, r.T_final, r.n_contrib):
            x.zero_()
        H.call("hyrf_rasterize", r._raster_args(), r.ws["r"])
        torch.cuda.synchronize()
        for a, b in zip((r.C_fg, r.T_final, r.n_contrib), ref):
            assert np.array_equal(np_(a), b)
    bad = np.arange(nt)
    bad[5] = nt + 7
    r.tile_order.copy_(torch.as_tensor(bad, dtype=torch.int32))
    r.status.zero_()
    H.call("hyrf_rasterize", r._raster_args(), r.ws["r"])
    torch.cuda.synchronize()
    assert H.read_status(r.status) & H.HYRF_ERR_BOUNDS


def test_separate_precull_and_depth_order_match_the_single_calls():
    """hyrf_precull + hyrf_query_fields(vis_ready=1) give the visible set
    and the field outputs of the single call bit for bit; hyrf_bin_sort with
    the depth order of hyrf_depth_order (computed from the positions, on the
    second stream in the pipeline) gives the instances and ranges of its own
    depth sort bit for bit."""
    w = synth.config3(n=30000, width=301, height=203, log2_T=15, n_clusters=32, precision="bf16",
                      table_init=0.3)
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg)
    assert r._overlap()
    r.fit_capacity()
    r.status.zero_()
    r.forward(None, want_keys=True)  # the split path: pre-cull, depth order beside the query
    torch.cuda.synchronize()
    assert H.read_status(r.status) == 0
    split = {k: np_(getattr(r, k)).copy() for k in ("vis_ids", "n_vis", "alpha", "scale", "quat", "color",
                                                      "vals", "ranges", "n_inst", "keys")}
    nv, K = int(split["n_vis"][0]), int(split["n_inst"][0])
    # the single calls
    H.hyrf_query_fields(ws=r.ws["q"], **r.query_kwargs())
    r.project()
    r._depth_ready = False
    r.bin_sort(want_keys=True)
    torch.cuda.synchronize()
    assert int(r.n_vis.item()) == nv and int(r.n_inst.item()) == K
    for k in ("vis_ids", "alpha", "scale", "quat", "color"):
        a = np_(getattr(r, k))
        assert np.array_equal(a[:nv], split[k][:nv]), k
    assert np.array_equal(np_(r.vals)[:K], split["vals"][:K])
    assert np.array_equal(np_(r.keys)[:K], split["keys"][:K])
    assert np.array_equal(np_(r.ranges), split["ranges"])


def test_view_with_every_gaussian_culled():
    """Edge case: the camera looks away from the scene, so the pre-cull keeps
    no Gaussian (n_vis = 0, K = 0). The step runs every stage on empty sets:
    the image is the background alone (against the oracle), no Gaussian
    receives a gradient, the background field does, and no status bit is
    set."""
    import dataclasses
    w = synth.config3(n=20000, width=161, height=113, log2_T=15, n_clusters=16, precision="bf16",
                      table_init=0.3)
    cam = w.cams[0]
    away = dataclasses.replace(cam, R=(np.diag([-1.0, 1.0, -1.0]) @ cam.R).astype(np.float32))
    w = dataclasses.replace(w, cams=[away])
    m = DeviceModel(w)
    r = ViewRenderer(m, away, w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
    tgt = cuda_f32(w.targets[0])
    r.set_capacity(1 << 16)
    r.status.zero_()
    m.zero_grad()
    r.forward(tgt, want_keys=False)
    r.backward()
    torch.cuda.synchronize()
    assert H.read_status(r.status) == 0
    assert int(r.n_vis.item()) == 0 and int(r.n_inst.item()) == 0
    assert np.all(np_(r.T_final) == 1.0) and np.all(np_(r.n_contrib) == 0) and np.all(np_(r.C_fg) == 0.0)
    fw = oracle.render(w.gaussians, w.fields, away, w.bg)
    assert np.abs(np_(r.C) - fw["C"]).max() < 4e-3
    for k in ("pos", "alpha_e", "scale_e", "color_e"):
        assert not np.any(np_(m.grad[k])), k
    assert np.any(np_(m.grad["rad_table"]))
