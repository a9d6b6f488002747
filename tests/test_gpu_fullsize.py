"""GPU parity at the full size of the headline workload: 1M Gaussians (256
clusters + 10 % far points), 1237x822, 16-level 2^19 BF16 grids, exact
background, through the same calls and launch configuration the benchmark
times (ViewRenderer with saved features).

The FP64 oracle cannot render this view in seconds, so each check uses what
it can compute exactly:
  * integers (visibility, rectangles, depth keys, the 15M-instance sort and
    the tile ranges) from the oracle's FP32 replay, bit for bit, over the
    whole view;
  * compositing forward and reverse over the whole image from stage inputs
    the oracle produced (its projection, its sort), on decision-safe pixels;
  * field query forward on a sample of visible Gaussians, and its reverse
    with upstream gradients that are non-zero on that sample only, so the
    oracle's sampled reverse is the exact expected value of every gradient
    buffer (tables and decoders included);
  * background forward on crops of the image (the oracle's camera shifted
    to each crop), and its reverse with dL/dC non-zero on the crops only.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2509_17083_gb300 import hyrf as H
from paper_2509_17083_gb300 import synth
from paper_2509_17083_gb300.pipeline import DeviceModel, ViewRenderer
from tests.gpu_util import (RELU_REPLAY_MARGIN_BF16, TOL_GRAD_BF16, TOL_GRAD_F32, TOL_IMG_F32, cuda_f32,
                             cuda_i32, np_, rel_l2)

pytestmark = pytest.mark.gpu

# the trained-like table spread used here
TABLE_INIT = 0.3
N_SAMPLE = 4096


@pytest.fixture(scope="module")
def scene():
    w = synth.config3(table_init=TABLE_INIT)
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
    tgt = cuda_f32(w.targets[0])
    r.fit_capacity(tgt)
    r.status.zero_()
    r.forward(tgt, want_keys=True)
    torch.cuda.synchronize()
    assert H.read_status(r.status) == 0
    ids = np.nonzero(oracle.precull_f32(w.gaussians.pos, w.cams[0]))[0].astype(np.int32)
    return w, m, r, ids


def test_fullsize_visibility_bit_exact(scene):
    w, m, r, ids = scene
    nv = int(r.n_vis.item())
    assert nv == len(ids) and nv > 900_000
    assert np.array_equal(np_(r.vis_ids)[:nv], ids)


def _stage_geometry(w, ids):
    """Projection inputs of the visible set from their own seeded generator:
    anisotropic scales e^U(-5,-2) and unit quaternions."""
    rng = np.random.default_rng(21)
    nv = len(ids)
    s = np.exp(rng.uniform(-5.0, -2.0, (nv, 3))).astype(np.float32)
    q = synth.random_quats(rng, nv)
    return w.gaussians.pos[ids].astype(np.float32), s, q


def _stage_opacity(nv):
    """Seeded opacities for the footprint (sigma of N(0, 1.5^2) logits)."""
    rng = np.random.default_rng(20)
    return (1.0 / (1.0 + np.exp(-1.5 * rng.standard_normal(nv)))).astype(np.float32)


def test_fullsize_project_and_bin_sort_bit_exact(scene):
    w, m, r, ids = scene
    cam = w.cams[0]
    pos, s, q = _stage_geometry(w, ids)
    nv = len(ids)
    op = _stage_opacity(nv)
    r.scale[:nv].copy_(cuda_f32(s))
    r.quat[:nv].copy_(cuda_f32(q))
    r.alpha[:nv].copy_(cuda_f32(op))
    r.status.zero_()
    r.project()
    r.bin_sort(want_keys=True)
    torch.cuda.synchronize()
    assert H.read_status(r.status) == 0
    rect, ntiles, depth, flag, m2, foot = oracle.project_f32_footprint(pos, s, q, cam, op)
    assert np.array_equal(np_(r.rect)[:nv], rect)
    assert np.array_equal(np_(r.ntiles)[:nv], ntiles)
    assert np.array_equal(np_(r.depth)[:nv].view(np.uint32), depth.view(np.uint32))
    assert np.array_equal(np_(r.flag)[:nv], flag)
    assert np.array_equal(np_(r.footprint)[:nv].view(np.uint32), foot.view(np.uint32))
    TX, TY = oracle.tiles_of(cam.width, cam.height)
    keys, vals, ranges = oracle.bin_sort(rect, depth, TX, TY, m2, foot)
    K = len(keys)
    assert int(r.n_inst.item()) == K and K > 5_000_000
    assert np.array_equal(np_(r.keys)[:K].view(np.uint64), keys)
    assert np.array_equal(np_(r.vals)[:K], vals)
    assert np.array_equal(np_(r.ranges), ranges)


def test_fullsize_rasterize_forward_and_reverse(scene):
    w, m, r, ids = scene
    cam = w.cams[0]
    W, H_ = cam.width, cam.height
    pos, s, q = _stage_geometry(w, ids)
    nv = len(ids)
    mean2d, conic, _ = oracle.project(pos.astype(np.float64), s.astype(np.float64), q.astype(np.float64),
                                      cam)
    rng = np.random.default_rng(22)
    op = 1.0 / (1.0 + np.exp(-rng.standard_normal(nv)))
    col = rng.uniform(0.0, 1.0, (nv, 3))
    # the instance lists the pipeline bins: opacity-aware footprints
    rect, _, depth, _, fm2, foot = oracle.project_f32_footprint(pos, s, q, cam, op.astype(np.float32))
    TX, TY = oracle.tiles_of(W, H_)
    _, vals, ranges = oracle.bin_sort(rect, depth, TX, TY, fm2, foot)
    m2, c2, op, col = [np.asarray(x, np.float32) for x in (mean2d, conic, op, col)]
    # the renderer's buffers carry these stage inputs through the same calls
    r.mean2d[:nv].copy_(cuda_f32(m2))
    r.conic[:nv].copy_(cuda_f32(c2))
    r.alpha[:nv].copy_(cuda_f32(op))
    r.color[:nv].copy_(cuda_f32(col))
    K = len(vals)
    r.vals[:K].copy_(cuda_i32(vals))
    r.ranges.copy_(cuda_i32(ranges))
    r.status.zero_()
    H.call("hyrf_rasterize", r._raster_args(), r.ws["r"])
    torch.cuda.synchronize()
    C, T, nc, mg = oracle.rasterize(W, H_, ranges, vals, m2, c2, op, col)
    safe = mg > 1e-4
    assert safe.mean() > 0.95, safe.mean()
    assert np.abs(np_(r.C_fg) - C)[safe].max() < TOL_IMG_F32
    assert np.abs(np_(r.T_final) - T)[safe].max() < TOL_IMG_F32
    assert np.array_equal(np_(r.n_contrib)[safe], nc[safe])
    # reverse, with dL/dC and dL/dT_final zero on unsafe pixels
    dC = (rng.standard_normal((H_, W, 3)) * safe[..., None]).astype(np.float32)
    dT = (rng.standard_normal((H_, W)) * safe).astype(np.float32)
    for t in (r.d_mean2d, r.d_conic, r.d_alpha, r.d_color):
        t.zero_()
    H.hyrf_rasterize_backward(r._raster_args(), ws=r.ws["rb"], d_C_fg=cuda_f32(dC), d_T_final=cuda_f32(dT),
                              d_mean2d=r.d_mean2d, d_conic=r.d_conic, d_alpha=r.d_alpha, d_color=r.d_color)
    torch.cuda.synchronize()
    rm, rc, ro, rcol = oracle.rasterize_backward(W, H_, ranges, vals, m2, c2, op, col, dC, dT)
    for gpu, ref, key in [(r.d_mean2d, rm, "mean2d"), (r.d_conic, rc, "conic"), (r.d_alpha, ro, "alpha"),
                          (r.d_color, rcol, "color")]:
        e = rel_l2(np_(gpu)[:nv], ref)
        assert e < TOL_GRAD_F32, (key, e)


def _sample(ids, seed, k=N_SAMPLE):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(len(ids), k, replace=False))


def test_fullsize_field_query_sampled(scene):
    w, m, r, ids = scene
    g = w.gaussians
    # the fixture's forward wrote the field outputs; later tests overwrite
    # them, so re-run the query alone
    fs = m.fields_struct()
    H.hyrf_query_fields(ws=r.ws["q"], n=m.n, pos=m.pos, alpha_e=m.alpha_e, scale_e=m.scale_e,
                        color_e=m.color_e, cam=r.ccam, fields=fs, vis_ids=r.vis_ids, n_vis=r.n_vis,
                        alpha=r.alpha, scale=r.scale, quat=r.quat, color=r.color, status=r.status,
                        features=r.feat_q)
    torch.cuda.synchronize()
    rows = _sample(ids, 23)
    sel = ids[rows]
    a, s, q, c = oracle.query_fields(g.pos[sel].astype(np.float64), g.alpha_e[sel], g.scale_e[sel],
                                     g.color_e[sel], w.cams[0], w.fields)
    for gpu, ref, tol in [(r.alpha, a, 5e-3), (r.scale, s, 5e-3), (r.quat, q, 2e-2), (r.color, c, 5e-3)]:
        err = np.abs(np_(gpu)[rows] - ref)
        assert err.max() < tol, err.max()
        assert err.mean() < tol / 10, err.mean()


def test_fullsize_field_query_reverse_sampled(scene):
    w, m, r, ids = scene
    g = w.gaussians
    cam = w.cams[0]
    nv = len(ids)
    # the oracle takes the decoders' ReLU branches as the BF16 kernels do;
    # rows with a replayed pre-activation near a kink are left out
    fr = oracle.replay_relu(w.fields, "bf16")
    rows = _sample(ids, 24, 2 * N_SAMPLE)
    sel = ids[rows]
    ok = oracle.relu_safe_mask(g, fr, cam, sel, RELU_REPLAY_MARGIN_BF16, RELU_REPLAY_MARGIN_BF16)
    rows, sel = rows[ok > 0], sel[ok > 0]
    assert len(rows) > 1.5 * N_SAMPLE, len(rows)
    rng = np.random.default_rng(25)
    up = [(rng.standard_normal((len(rows),) + sh) * 1e-3).astype(np.float32)
          for sh in [(), (3,), (4,), (3,)]]
    # forward first (restores the field outputs and the saved features)
    fs = m.fields_struct()
    H.hyrf_query_fields(ws=r.ws["q"], n=m.n, pos=m.pos, alpha_e=m.alpha_e, scale_e=m.scale_e,
                        color_e=m.color_e, cam=r.ccam, fields=fs, vis_ids=r.vis_ids, n_vis=r.n_vis,
                        alpha=r.alpha, scale=r.scale, quat=r.quat, color=r.color, status=r.status,
                        features=r.feat_q)
    for t, u in zip((r.d_alpha, r.d_scale, r.d_quat, r.d_color), up):
        t.zero_()
        t[torch.as_tensor(rows, device=t.device)] = cuda_f32(u)
    m.zero_grad()
    r.status.zero_()
    r.backward_fields()
    torch.cuda.synchronize()
    assert H.read_status(r.status) == 0
    ref = oracle.query_fields_backward(g.pos[sel].astype(np.float64), g.alpha_e[sel], g.scale_e[sel],
                                       g.color_e[sel], cam, fr, *[u.astype(np.float64) for u in up])
    full = {k: np.zeros(np.asarray(getattr(g, k)).shape) for k in ("pos", "alpha_e", "scale_e", "color_e")}
    for k in full:
        full[k][sel] = ref[k]
    for k in ("pos", "alpha_e", "scale_e", "color_e"):
        e = rel_l2(np_(m.grad[k]), full[k])
        assert e < TOL_GRAD_BF16, (k, e)
    for k in ("geo_table", "rad_table"):
        e = rel_l2(np_(m.grad[k]), ref[k])
        assert e < TOL_GRAD_BF16, (k, e)
    for k in ("geo_W", "col_W", "geo_b", "col_b"):
        for l in range(3):
            e = rel_l2(np_(m.grad[k][l]), ref[k][l])
            assert e < TOL_GRAD_BF16, (k, l, e)
    assert nv == int(r.n_vis.item())


def _crop(cam, x0, y0, cw, ch):
    return dataclasses.replace(cam, cx=cam.cx - x0, cy=cam.cy - y0, width=cw, height=ch)


def test_fullsize_background_crops(scene):
    w, m, r, ids = scene
    cam = w.cams[0]
    W, H_ = cam.width, cam.height
    rng = np.random.default_rng(26)
    Cfg = rng.uniform(0, 1, (H_, W, 3)).astype(np.float32)
    T = rng.uniform(0, 1, (H_, W)).astype(np.float32)
    r.C_fg.copy_(cuda_f32(Cfg))
    r.T_final.copy_(cuda_f32(T))
    r.status.zero_()
    H.call("hyrf_composite_background", r._bg_args(), r.ws["b"])
    torch.cuda.synchronize()
    Cg = np_(r.C)
    # 8 disjoint 48x40 crops, one per cell of a 4 x 2 grid, jittered
    cw, ch = 48, 40
    crops = [(int(i * (W // 4) + rng.integers(0, W // 4 - cw)), int(j * (H_ // 2) + rng.integers(0, H_ // 2 - ch)))
             for i in range(4) for j in range(2)]
    dC = np.zeros((H_, W, 3), np.float32)
    fr = oracle.replay_relu(w.fields, "bf16")
    kept = []
    for (x0, y0) in crops:
        cc = _crop(cam, x0, y0, cw, ch)
        C, _ = oracle.background(cc, w.fields, w.bg, Cfg[y0:y0 + ch, x0:x0 + cw], T[y0:y0 + ch, x0:x0 + cw])
        assert np.abs(Cg[y0:y0 + ch, x0:x0 + cw] - C).max() < 2e-3  # bf16 decoder
        safe = oracle.bg_margins(cc, fr, w.bg) > RELU_REPLAY_MARGIN_BF16
        kept.append(safe.mean())
        dC[y0:y0 + ch, x0:x0 + cw] = rng.standard_normal((ch, cw, 3)) * safe[..., None]
    assert np.mean(kept) > 0.75, kept
    r.dC.copy_(cuda_f32(dC))
    m.zero_grad()
    H.hyrf_composite_background_backward(r._bg_args(), ws=r.ws["bb"], d_C=r.dC, d_C_fg=None,
                                         d_T_final=r.dT, grads=m.grads_struct(), loss_scale=r.loss_scale)
    torch.cuda.synchronize()
    assert H.read_status(r.status) == 0
    tab, cW, cb = None, None, None
    for (x0, y0) in crops:
        cc = _crop(cam, x0, y0, cw, ch)
        ref = oracle.background_backward(cc, fr, w.bg, T[y0:y0 + ch, x0:x0 + cw],
                                         dC[y0:y0 + ch, x0:x0 + cw])
        e = np.abs(np_(r.dT)[y0:y0 + ch, x0:x0 + cw] - ref["T_final"]).max()
        assert e < 2e-3 * max(1.0, np.abs(ref["T_final"]).max()), e
        if tab is None:
            tab, cW, cb = ref["rad_table"], ref["col_W"], ref["col_b"]
        else:
            tab = tab + ref["rad_table"]
            cW = [x + y for x, y in zip(cW, ref["col_W"])]
            cb = [x + y for x, y in zip(cb, ref["col_b"])]
    assert rel_l2(np_(m.grad["rad_table"]), tab) < TOL_GRAD_BF16
    for l in range(3):
        assert rel_l2(np_(m.grad["col_W"][l]), cW[l]) < TOL_GRAD_BF16
        assert rel_l2(np_(m.grad["col_b"][l]), cb[l]) < TOL_GRAD_BF16
