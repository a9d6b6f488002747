"""The Tab. 5 ablation paths against the oracle: explicit-only (the oracle
with zero tables and decoder weights, whose geometry bias gives alpha_n =
s_n = 0 and rotation (1,0,0,0), colour bias 0), neural-only (explicit parts
zero), one grid for both decoders (the oracle with the geometry grid set to
the radiance grid), and no background (C = C_fg)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2509_17083_gb300 import hyrf as H
from paper_2509_17083_gb300 import synth
from paper_2509_17083_gb300.pipeline import DeviceModel, ViewRenderer
from tests.gpu_util import TOL_GRAD_F32, TOL_Q_F32_TRAINED, np_, rel_l2

pytestmark = pytest.mark.gpu


def _w(**kw):
    return synth.config2(n=6000, width=150, height=120, log2_T=12, n_clusters=16, table_init=0.3, seed=9, **kw)


def _query(w, model_kw=None, **kw):
    m = DeviceModel(w, **(model_kw or {}))
    r = ViewRenderer(m, w.cams[0], w.bg, **kw)
    H.hyrf_query_fields(ws=r.ws["q"], **r.query_kwargs())
    torch.cuda.synchronize()
    nv = int(r.n_vis.item())
    ids = np.nonzero(oracle.precull_f32(w.gaussians.pos, w.cams[0]))[0]
    assert nv == len(ids)
    return m, r, ids, nv


def _cmp(r, nv, ref, tol):
    for gpu, x in zip((r.alpha, r.scale, r.quat, r.color), ref):
        assert np.abs(np_(gpu)[:nv] - x).max() < tol


def test_explicit_only_equals_fieldless_oracle():
    w = _w()
    m, r, ids, nv = _query(w, neural=False)
    g = w.gaussians
    fl = w.fields
    zero = dataclasses.replace(
        fl, geo=dataclasses.replace(fl.geo, table=np.zeros_like(fl.geo.table)),
        rad=dataclasses.replace(fl.rad, table=np.zeros_like(fl.rad.table)),
        geo_mlp=dataclasses.replace(fl.geo_mlp, W=[np.zeros_like(x) for x in fl.geo_mlp.W]),
        col_mlp=dataclasses.replace(fl.col_mlp, W=[np.zeros_like(x) for x in fl.col_mlp.W],
                                    b=[np.zeros_like(x) for x in fl.col_mlp.b]))
    ref = oracle.query_fields(g.pos[ids].astype(np.float64), g.alpha_e[ids], g.scale_e[ids], g.color_e[ids],
                              w.cams[0], zero)
    _cmp(r, nv, ref, 2e-6)
    # reverse: explicit gradients only
    rng = np.random.default_rng(3)
    ups = [torch.tensor(rng.standard_normal(t[:nv].shape).astype(np.float32), device="cuda")
           for t in (r.d_alpha, r.d_scale, r.d_quat, r.d_color)]
    for t, u in zip((r.d_alpha, r.d_scale, r.d_quat, r.d_color), ups):
        t[:nv] = u
    m.zero_grad()
    r.backward_fields()
    torch.cuda.synchronize()
    refg = oracle.query_fields_backward(g.pos[ids].astype(np.float64), g.alpha_e[ids], g.scale_e[ids],
                                        g.color_e[ids], w.cams[0], zero, *[np_(u).astype(np.float64) for u in ups])
    for k in ("alpha_e", "scale_e", "color_e"):
        full = np.zeros(np.asarray(getattr(g, k)).shape)
        full[ids] = refg[k]
        assert rel_l2(np_(m.grad[k]), full) < TOL_GRAD_F32, k
    assert float(m.grad["geo_table"].abs().max()) == 0.0 and float(m.grad["rad_table"].abs().max()) == 0.0


def test_neural_only_equals_zero_explicit_oracle():
    w = _w()
    m, r, ids, nv = _query(w, explicit=False)
    g = w.gaussians
    z = np.zeros(len(ids), np.float32)
    ref = oracle.query_fields(g.pos[ids].astype(np.float64), z, z, np.zeros((len(ids), 3), np.float32), w.cams[0],
                              w.fields)
    _cmp(r, nv, ref, TOL_Q_F32_TRAINED)


def test_single_grid_equals_oracle_with_shared_grid():
    w = _w()
    m, r, ids, nv = _query(w, model_kw=dict(coupled=True))
    g = w.gaussians
    shared = dataclasses.replace(w.fields, geo=w.fields.rad)
    ref = oracle.query_fields(g.pos[ids].astype(np.float64), g.alpha_e[ids], g.scale_e[ids], g.color_e[ids],
                              w.cams[0], shared)
    _cmp(r, nv, ref, TOL_Q_F32_TRAINED)


def test_no_background_is_foreground():
    w = _w()
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg, background=False)
    r.fit_capacity()
    r.forward(None)
    torch.cuda.synchronize()
    assert torch.equal(r.C, r.C_fg)
    r.dC.normal_()
    H.hyrf_composite_background_backward(r._bg_args(), ws=r.ws["bb"], d_C=r.dC, d_C_fg=r.C, d_T_final=r.dT,
                                         grads=m.grads_struct(), loss_scale=1.0)
    torch.cuda.synchronize()
    assert torch.equal(r.C, r.dC) and float(r.dT.abs().max()) == 0.0


def test_no_precull_queries_every_gaussian_and_projection_drops_the_rest():
    w = synth.config3_360(n=8000, width=200, height=150, log2_T=14, n_clusters=16, precision="f32")
    cam = w.cams[0]
    m = DeviceModel(w)
    r = ViewRenderer(m, cam, w.bg, precull=False)
    r.fit_capacity()
    r.forward(None)
    torch.cuda.synchronize()
    n = w.gaussians.n
    assert int(r.n_vis.item()) == n
    assert np.array_equal(np_(r.vis_ids)[:n], np.arange(n))
    rng = np.random.default_rng(8)
    s = np.exp(rng.uniform(-5, -2, (n, 3))).astype(np.float32)
    q = synth.random_quats(rng, n)
    op = (1.0 / (1.0 + np.exp(-rng.standard_normal(n)))).astype(np.float32)
    r.scale[:n].copy_(torch.tensor(s, device="cuda"))
    r.quat[:n].copy_(torch.tensor(q, device="cuda"))
    r.alpha[:n].copy_(torch.tensor(op, device="cuda"))
    r.project()
    torch.cuda.synchronize()
    rect, ntiles, depth, flag, _, _ = oracle.project_f32_footprint(w.gaussians.pos, s, q, cam, op)
    assert np.array_equal(np_(r.rect)[:n], rect) and np.array_equal(np_(r.ntiles)[:n], ntiles)
    behind = depth <= cam.z_near
    assert behind.sum() > n // 4 and (ntiles[behind] == 0).all()
