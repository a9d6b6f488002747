"""GPU parity of each stage of the C ABI against the FP64 oracle.

Every stage is fed inputs produced by the seeded generators or by the
oracle itself (never by the CUDA path), so a failure localises to one
stage. Integer outputs (visibility, rectangles, sort keys, ranges) must be
bit-exact; floating outputs meet the FP32 tolerances in gpu_util.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_17083_gb300 import hyrf as H
from paper_2509_17083_gb300 import synth
from paper_2509_17083_gb300.pipeline import DeviceModel, ViewRenderer
from tests.gpu_util import (TOL_GRAD_F32, TOL_IMG_F32, TOL_Q_F32, TOL_Q_F32_TRAINED, cuda_f32,
                            cuda_i32, np_, rel_l2)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return H.lib()


def _cfg(name):
    init = 0.5 if name.endswith("_trained") else 1e-4
    if name.startswith("c1"):
        return synth.config1(n=3000, width=100, height=84, table_init=init, seed=4)
    if name.startswith("c2"):
        return synth.config2(n=6000, width=150, height=120, log2_T=12, n_clusters=16,
                             table_init=init, seed=5)
    raise KeyError(name)


# ------------------------------------------------------------------ pre-cull + query

@pytest.mark.parametrize("name", ["c1", "c2"])
def test_precull_compaction_bit_exact(lib, name):
    w = _cfg(name)
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg)
    r.forward()
    torch.cuda.synchronize()
    vis = oracle.precull_f32(w.gaussians.pos, w.cams[0])
    ids = np.nonzero(vis)[0]
    nv = int(r.n_vis.item())
    assert nv == len(ids)
    assert np.array_equal(np_(r.vis_ids)[:nv], ids)
    assert H.read_status(r.status) == 0


@pytest.mark.parametrize("name", ["c1", "c2", "c1_trained", "c2_trained"])
def test_query_fields_matches_oracle(lib, name):
    w = _cfg(name)
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg)
    r.forward()
    torch.cuda.synchronize()
    g = w.gaussians
    ids = np.nonzero(oracle.precull_f32(g.pos, w.cams[0]))[0]
    a, s, q, c = oracle.query_fields(g.pos[ids].astype(np.float64), g.alpha_e[ids], g.scale_e[ids],
                                     g.color_e[ids], w.cams[0], w.fields)
    nv = len(ids)
    tol = TOL_Q_F32_TRAINED if name.endswith("_trained") else TOL_Q_F32
    for gpu, ref in [(r.alpha, a), (r.scale, s), (r.quat, q), (r.color, c)]:
        err = np.abs(np_(gpu)[:nv] - ref).max()
        assert err < tol, err


# ------------------------------------------------------------------ projection

def _proj_inputs(rng, n, cam):
    pos = np.stack([rng.uniform(-2.5, 2.5, n), rng.uniform(-1.8, 1.8, n), rng.uniform(0.5, 8, n)], 1)
    s = np.exp(rng.uniform(-5, -0.5, (n, 3)))
    q = synth.random_quats(rng, n) * rng.uniform(0.2, 3, (n, 1))
    deg = rng.choice(n, n // 50, replace=False)  # near-degenerate: anisotropy 1e4
    s[deg] = np.array([1e-1, 1e-5, 1e-5])
    return pos.astype(np.float32), s.astype(np.float32), q.astype(np.float32)


def test_project_bit_exact_integers_and_fp64_floats(lib):
    rng = np.random.default_rng(11)
    cam = synth.look_at([0.4, -0.3, -1.0], [0, 0, 4], 333, 211, 65.0)
    n = 20000
    pos, s, q = _proj_inputs(rng, n, cam)
    dev = "cuda"
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    nv = torch.tensor([n], dtype=torch.int32, device=dev)
    out = dict(mean2d=torch.zeros(n, 2, device=dev), conic=torch.zeros(n, 3, device=dev),
               depth=torch.zeros(n, device=dev), rect=torch.zeros(n, 4, dtype=torch.int32, device=dev),
               ntiles=torch.zeros(n, dtype=torch.int32, device=dev),
               fp64_flag=torch.zeros(n, dtype=torch.uint8, device=dev))
    # all z > 0 here: pre-cull is not involved, projection alone
    H.hyrf_project(n=n, pos=cuda_f32(pos), vis_ids=ids, n_vis=nv, scale=cuda_f32(s), quat=cuda_f32(q),
                   cam=H.camera(cam), tile=16, **out)
    torch.cuda.synchronize()
    rect, ntiles, depth, flag = oracle.project_f32(pos, s, q, cam)
    assert np.array_equal(np_(out["rect"]), rect)
    assert np.array_equal(np_(out["ntiles"]), ntiles)
    assert np.array_equal(np_(out["depth"]).view(np.uint32), depth.view(np.uint32))
    assert np.array_equal(np_(out["fp64_flag"]), flag)
    assert flag.sum() > 0  # the FP64 branch ran
    m, c, d = oracle.project(pos.astype(np.float64), s.astype(np.float64), q.astype(np.float64), cam)
    np.testing.assert_allclose(np_(out["mean2d"]), m, rtol=2e-6, atol=1e-3)
    # conic, relative to its own scale: FP32 inversion where |det| >= 1e-2 a c
    # (cancellation amplifies the ~20-op rounding of Sigma' by up to 100x),
    # FP64 inversion below
    cg = np_(out["conic"]).astype(np.float64)
    scale = np.abs(c).max(1, keepdims=True)
    err = (np.abs(cg - c) / scale).max(1)
    assert np.quantile(err[flag == 0], 0.999) < 1e-4 and err[flag == 0].max() < 2e-3, err.max()
    assert err[flag == 1].max() < 1e-5, err[flag == 1].max()


def _footprint_scene(kind, rng, n, cam):
    pos, s, q = _proj_inputs(rng, n, cam)
    s[:, 0] *= np.exp(rng.uniform(0.0, 2.5, n)).astype(np.float32)  # anisotropic
    op = (1.0 / (1.0 + np.exp(-1.5 * rng.standard_normal(n)))).astype(np.float32)
    if kind == "tall":
        # thin, faint, mostly upright Gaussians: many rectangle rows whose
        # ellipse misses them (more tile rows than instances per expansion CTA)
        s[:] = np.array([0.004, 0.6, 0.004], np.float32) * rng.uniform(0.5, 1.5, (n, 1)).astype(np.float32)
        q = np.concatenate([np.ones((n, 1)), rng.normal(0.0, 0.01, (n, 3))], 1).astype(np.float32)
        op = rng.uniform(0.0045, 0.01, n).astype(np.float32)
    elif kind == "sparse":
        # most Gaussians below 1/255: many zero-instance Gaussians per CTA range
        op[rng.random(n) < 0.995] = 1.0 / 300.0
    elif kind == "big":
        # a few large Gaussians: rectangles of more than 16 tile rows, whose
        # footprint records carry no packed spans
        big = rng.random(n) < 0.01
        s[big] *= 12.0
    op[:50] = 1.0 / 300.0  # below 1/255: no footprint
    return pos, s, q, op


@pytest.mark.parametrize("kind", ["mixed", "tall", "sparse", "big"])
def test_project_footprint_and_bin_sort_bit_exact(lib, kind):
    """The binning's opacity-aware footprint: the projection's tile counts
    and footprint records, and the instance lists hyrf_bin_sort emits from
    them, bit for bit against the oracle's FP32 replay. "mixed" takes the
    expansion's packed-span path; "tall" and "big" (rectangles of more than
    16 tile rows) its row-parallel path, "tall" also beyond the rows a CTA
    caches; "sparse" (more Gaussians per CTA range than it caches) the
    per-Gaussian path."""
    rng = np.random.default_rng(14)
    H_ = {"mixed": 211, "tall": 420, "sparse": 211, "big": 420}[kind]
    cam = synth.look_at([0.4, -0.3, -1.0], [0, 0, 4], 333, H_, 65.0)
    n = {"mixed": 20000, "tall": 12000, "sparse": 120000, "big": 20000}[kind]
    pos, s, q, op = _footprint_scene(kind, rng, n, cam)
    dev = "cuda"
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    nv = torch.tensor([n], dtype=torch.int32, device=dev)
    out = dict(mean2d=torch.zeros(n, 2, device=dev), conic=torch.zeros(n, 3, device=dev),
               depth=torch.zeros(n, device=dev), rect=torch.zeros(n, 4, dtype=torch.int32, device=dev),
               ntiles=torch.zeros(n, dtype=torch.int32, device=dev),
               fp64_flag=torch.zeros(n, dtype=torch.uint8, device=dev), footprint=torch.zeros(n, 12, device=dev))
    H.hyrf_project(n=n, pos=cuda_f32(pos), vis_ids=ids, n_vis=nv, scale=cuda_f32(s), quat=cuda_f32(q),
                   cam=H.camera(cam), tile=16, alpha=cuda_f32(op), **out)
    torch.cuda.synchronize()
    rect, ntiles, depth, flag, m2, foot = oracle.project_f32_footprint(pos, s, q, cam, op)
    assert np.array_equal(np_(out["rect"]), rect)
    assert np.array_equal(np_(out["ntiles"]), ntiles)
    assert np.array_equal(np_(out["fp64_flag"]), flag)
    assert np.array_equal(np_(out["footprint"]).view(np.uint32), foot.view(np.uint32))
    assert np.array_equal(np_(out["mean2d"]).view(np.uint32), m2.view(np.uint32))
    area = np.where(rect[:, 2] > rect[:, 0], (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1]), 0)
    assert ntiles.sum() < 0.9 * area.sum() and (ntiles[:50] == 0).all()
    rows = np.where(rect[:, 2] > rect[:, 0], rect[:, 3] - rect[:, 1], 0)
    if kind == "tall":
        assert rows.sum() > 1.5 * ntiles.sum(), (rows.sum(), ntiles.sum())
    if kind == "sparse":
        assert (ntiles == 0).sum() > 100 * (ntiles > 0).sum()
    unpacked = (rows > 16) | (rect[:, 2] - rect[:, 0] > 255)
    if kind in ("tall", "big"):
        assert unpacked.sum() > 20
    else:
        assert not unpacked.any()
    TX, TY = oracle.tiles_of(cam.width, cam.height)
    keys, vals, ranges = oracle.bin_sort(rect, depth, TX, TY, m2, foot)
    K = len(keys)
    got = dict(keys=torch.zeros(K + 8, dtype=torch.int64, device=dev),
               vals=torch.zeros(K + 8, dtype=torch.int32, device=dev),
               ranges=torch.zeros(TX * TY, 2, dtype=torch.int32, device=dev),
               n_instances=torch.zeros(1, dtype=torch.int32, device=dev),
               status=torch.zeros(1, dtype=torch.int32, device=dev))
    H.hyrf_bin_sort(n=n, n_vis=nv, rect=out["rect"], ntiles=out["ntiles"], depth=out["depth"], tiles_x=TX,
                    tiles_y=TY, capacity=K + 8, mean2d=out["mean2d"], footprint=out["footprint"], **got)
    torch.cuda.synchronize()
    assert H.read_status(got["status"]) == 0
    assert int(got["n_instances"].item()) == K
    assert np.array_equal(np_(got["keys"])[:K].view(np.uint64), keys)
    assert np.array_equal(np_(got["vals"])[:K], vals)
    assert np.array_equal(np_(got["ranges"]), ranges)
    # mean2d and footprint go together
    with pytest.raises(H.HyrfError):
        H.hyrf_bin_sort(n=n, n_vis=nv, rect=out["rect"], ntiles=out["ntiles"], depth=out["depth"], tiles_x=TX,
                        tiles_y=TY, capacity=K + 8, footprint=out["footprint"], **got)


def test_project_backward_matches_oracle(lib):
    rng = np.random.default_rng(12)
    cam = synth.look_at([0.4, -0.3, -1.0], [0, 0, 4], 160, 120, 65.0)
    n = 4000
    pos, s, q = _proj_inputs(rng, n, cam)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    dm, dc = rng.standard_normal((n, 2)), rng.standard_normal((n, 3)) * 0.01
    dev = "cuda"
    d_pos = torch.zeros(n, 3, device=dev)
    d_s, d_q = torch.zeros(n, 3, device=dev), torch.zeros(n, 4, device=dev)
    H.hyrf_project_backward(n=n, pos=cuda_f32(pos), vis_ids=torch.arange(n, dtype=torch.int32, device=dev),
                            n_vis=torch.tensor([n], dtype=torch.int32, device=dev), scale=cuda_f32(s),
                            quat=cuda_f32(q), cam=H.camera(cam), d_mean2d=cuda_f32(dm),
                            d_conic=cuda_f32(dc), d_pos=d_pos, d_scale=d_s, d_quat=d_q)
    torch.cuda.synchronize()
    rp, rs, rq = oracle.project_backward(pos.astype(np.float64), s.astype(np.float64),
                                         q.astype(np.float64), cam, dm.astype(np.float32).astype(np.float64),
                                         dc.astype(np.float32).astype(np.float64))
    # exclude the near-degenerate Gaussians from the FP32 relative check, then
    # check them separately (FP64 inverse derivative)
    _, _, _, flag = oracle.project_f32(pos, s, q, cam)
    ok = flag == 0
    for gpu, ref in [(d_pos, rp), (d_s, rs), (d_q, rq)]:
        assert rel_l2(np_(gpu)[ok], ref[ok]) < TOL_GRAD_F32
        assert rel_l2(np_(gpu)[~ok], ref[~ok]) < 1e-2


# ------------------------------------------------------------------ binning

@pytest.mark.parametrize("W,H_,n", [(64, 48, 500), (333, 211, 20000), (1237, 822, 60000)])
def test_bin_sort_bit_exact(lib, W, H_, n):
    rng = np.random.default_rng(W)
    cam = synth.pinhole(W, H_, 60.0)
    pos, s, q = _proj_inputs(rng, n, cam)
    rect, ntiles, depth, _ = oracle.project_f32(pos, s, q, cam)
    # ties: copy some depths so equal keys occur
    depth[: n // 10] = depth[n // 10: 2 * (n // 10)]
    TX, TY = oracle.tiles_of(W, H_)
    keys, vals, ranges = oracle.bin_sort(rect, depth, TX, TY)
    K = len(keys)
    dev = "cuda"
    cap = K + 1000
    out_keys = torch.zeros(cap, dtype=torch.int64, device=dev)
    out_vals = torch.zeros(cap, dtype=torch.int32, device=dev)
    out_ranges = torch.zeros(TX * TY, 2, dtype=torch.int32, device=dev)
    n_inst = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    H.hyrf_bin_sort(n=n, n_vis=torch.tensor([n], dtype=torch.int32, device=dev), rect=cuda_i32(rect),
                    ntiles=cuda_i32(ntiles), depth=cuda_f32(depth), tiles_x=TX, tiles_y=TY,
                    capacity=cap, keys=out_keys, vals=out_vals, ranges=out_ranges,
                    n_instances=n_inst, status=status)
    torch.cuda.synchronize()
    assert int(n_inst.item()) == K
    assert np.array_equal(np_(out_keys)[:K].view(np.uint64), keys)
    assert np.array_equal(np_(out_vals)[:K], vals)
    assert np.array_equal(np_(out_ranges), ranges)
    assert H.read_status(status) == 0


def test_bin_sort_overflow_sets_status(lib):
    rng = np.random.default_rng(3)
    cam = synth.pinhole(200, 120, 60.0)
    n = 3000
    pos, s, q = _proj_inputs(rng, n, cam)
    rect, ntiles, depth, _ = oracle.project_f32(pos, s, q, cam)
    TX, TY = oracle.tiles_of(200, 120)
    K = int(ntiles.sum())
    cap = K // 2
    dev = "cuda"
    vals = torch.zeros(cap, dtype=torch.int32, device=dev)
    ranges = torch.zeros(TX * TY, 2, dtype=torch.int32, device=dev)
    n_inst = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    H.hyrf_bin_sort(n=n, n_vis=torch.tensor([n], dtype=torch.int32, device=dev), rect=cuda_i32(rect),
                    ntiles=cuda_i32(ntiles), depth=cuda_f32(depth), tiles_x=TX, tiles_y=TY,
                    capacity=cap, keys=None, vals=vals, ranges=ranges, n_instances=n_inst,
                    status=status)
    st = H.read_status(status)
    assert st & H.HYRF_ERR_OVERFLOW
    assert int(n_inst.item()) == cap
    # every written instance is a valid index; ranges stay inside the capacity
    v = np_(vals)
    assert v.min() >= 0 and v.max() < n
    assert np_(ranges).max() <= cap


def test_invalid_arguments_rejected_on_host(lib):
    with pytest.raises(H.HyrfError):
        H.hyrf_project(n=-1, tile=16)
    with pytest.raises(H.HyrfError):
        H.hyrf_rasterize(n=1, width=16, height=16, tile=8)


# ------------------------------------------------------------------ compositing

def _raster_scene(rng, W, H_, n):
    cam = synth.pinhole(W, H_, 60.0)
    pos = np.stack([rng.uniform(-2, 2, n), rng.uniform(-1.3, 1.3, n), rng.uniform(2, 6, n)], 1)
    s = np.exp(rng.uniform(-4.5, -1.8, (n, 3)))
    q = synth.random_quats(rng, n)
    pos, s, q = pos.astype(np.float32), s.astype(np.float32), q.astype(np.float32)
    m, c, _ = oracle.project(pos.astype(np.float64), s.astype(np.float64), q.astype(np.float64), cam)
    rect, ntiles, depth, _ = oracle.project_f32(pos, s, q, cam)
    TX, TY = oracle.tiles_of(W, H_)
    keys, vals, ranges = oracle.bin_sort(rect, depth, TX, TY)
    op = (1 / (1 + np.exp(-rng.standard_normal(n) - 0.5)))
    op[: n // 20] = 0.999  # alpha clamped at 0.99
    col = rng.uniform(0, 1, (n, 3))
    # the FP32 values both sides use
    m, c, op, col = [np.asarray(x, np.float32) for x in (m, c, op, col)]
    return cam, m, c, op, col, vals, ranges


def _gpu_raster(n, W, H_, m, c, op, col, vals, ranges):
    dev = "cuda"
    args = dict(n=n, n_vis=torch.tensor([n], dtype=torch.int32, device=dev), ranges=cuda_i32(ranges),
                vals=cuda_i32(vals), mean2d=cuda_f32(m), conic=cuda_f32(c), alpha=cuda_f32(op),
                color=cuda_f32(col), width=W, height=H_, tile=16,
                C_fg=torch.zeros(H_, W, 3, device=dev), T_final=torch.zeros(H_, W, device=dev),
                n_contrib=torch.zeros(H_, W, dtype=torch.int32, device=dev))
    a = H._fill(H.hyrf_rasterize_args(), args)
    H.call("hyrf_rasterize", a)
    return a, args


@pytest.mark.parametrize("W,H_,n", [(70, 50, 400), (257, 191, 8000)])
def test_rasterize_matches_oracle(lib, W, H_, n):
    rng = np.random.default_rng(W + n)
    cam, m, c, op, col, vals, ranges = _raster_scene(rng, W, H_, n)
    a, args = _gpu_raster(n, W, H_, m, c, op, col, vals, ranges)
    torch.cuda.synchronize()
    C, T, nc, mg = oracle.rasterize(W, H_, ranges, vals, m, c, op, col)
    safe = mg > 1e-4  # pixels with no threshold test within 1e-4 (relative) of its threshold
    assert safe.mean() > 0.98
    Cg, Tg, ncg = np_(args["C_fg"]), np_(args["T_final"]), np_(args["n_contrib"])
    assert np.abs(Cg - C)[safe].max() < TOL_IMG_F32
    assert np.abs(Tg - T)[safe].max() < TOL_IMG_F32
    assert np.array_equal(ncg[safe], nc[safe])


@pytest.mark.parametrize("W,H_,n", [(70, 50, 400), (257, 191, 8000)])
def test_rasterize_backward_matches_oracle(lib, W, H_, n):
    rng = np.random.default_rng(W + n + 1)
    cam, m, c, op, col, vals, ranges = _raster_scene(rng, W, H_, n)
    a, args = _gpu_raster(n, W, H_, m, c, op, col, vals, ranges)
    _, _, _, mg = oracle.rasterize(W, H_, ranges, vals, m, c, op, col)
    safe = (mg > 1e-4).astype(np.float32)
    dC = (rng.standard_normal((H_, W, 3)) * safe[..., None]).astype(np.float32)
    dT = (rng.standard_normal((H_, W)) * safe).astype(np.float32)
    dev = "cuda"
    g = dict(d_mean2d=torch.zeros(n, 2, device=dev), d_conic=torch.zeros(n, 3, device=dev),
             d_alpha=torch.zeros(n, device=dev), d_color=torch.zeros(n, 3, device=dev))
    H.hyrf_rasterize_backward(a, d_C_fg=cuda_f32(dC), d_T_final=cuda_f32(dT), **g)
    torch.cuda.synchronize()
    rm, rc, ro, rcol = oracle.rasterize_backward(W, H_, ranges, vals, m, c, op, col, dC, dT)
    for key, ref in [("d_mean2d", rm), ("d_conic", rc), ("d_alpha", ro), ("d_color", rcol)]:
        e = rel_l2(np_(g[key]), ref)
        assert e < TOL_GRAD_F32, (key, e)


def test_rasterize_records_shared_by_forward_and_reverse(lib):
    """The optional records buffer: the forward packs the records into it
    and the reverse reads them instead of packing again; the image, T_final
    and n_contrib equal those of the calls without it bit for bit, the
    gradients up to the order of their atomic sums."""
    rng = np.random.default_rng(77)
    W, H_, n = 181, 133, 3000
    cam, m, c, op, col, vals, ranges = _raster_scene(rng, W, H_, n)
    dev = "cuda"
    a0, args0 = _gpu_raster(n, W, H_, m, c, op, col, vals, ranges)
    rec = torch.full((n, 12), float("nan"), device=dev)  # must be overwritten by the forward
    args1 = dict(args0, C_fg=torch.zeros(H_, W, 3, device=dev), T_final=torch.zeros(H_, W, device=dev),
                 n_contrib=torch.zeros(H_, W, dtype=torch.int32, device=dev), records=rec)
    a1 = H._fill(H.hyrf_rasterize_args(), args1)
    H.call("hyrf_rasterize", a1)
    dC = rng.standard_normal((H_, W, 3)).astype(np.float32)
    dT = rng.standard_normal((H_, W)).astype(np.float32)
    outs = []
    for a in (a0, a1):
        g = dict(d_mean2d=torch.zeros(n, 2, device=dev), d_conic=torch.zeros(n, 3, device=dev),
                 d_alpha=torch.zeros(n, device=dev), d_color=torch.zeros(n, 3, device=dev))
        H.hyrf_rasterize_backward(a, d_C_fg=cuda_f32(dC), d_T_final=cuda_f32(dT), **g)
        outs.append(g)
    torch.cuda.synchronize()
    for k in ("C_fg", "T_final", "n_contrib"):
        assert np.array_equal(np_(args0[k]), np_(args1[k])), k
    # the gradients are sums of float atomics, whose order varies from run to
    # run: equal up to that rounding
    for k in outs[0]:
        assert rel_l2(np_(outs[1][k]), np_(outs[0][k])) < 1e-6, k
    assert not np.isnan(np_(rec)).any()
    # a misaligned records pointer is refused
    bad = dict(args1, records=torch.zeros(n * 12 + 1, device=dev)[1:])
    with pytest.raises(H.HyrfError):
        H.call("hyrf_rasterize", H._fill(H.hyrf_rasterize_args(), bad))


# ------------------------------------------------------------------ background and loss

@pytest.mark.parametrize("mode", [0, 1])
def test_background_matches_oracle(lib, mode):
    w = synth.config1(n=10, width=90, height=70, table_init=0.5, seed=6)
    w.bg = synth.Background(mode, 12, 20)
    cam = w.cams[0]
    rng = np.random.default_rng(7)
    Cfg = rng.uniform(0, 1, (70, 90, 3)).astype(np.float32)
    T = rng.uniform(0, 1, (70, 90)).astype(np.float32)
    m = DeviceModel(w)
    r = ViewRenderer(m, cam, w.bg)
    r.C_fg.copy_(cuda_f32(Cfg))
    r.T_final.copy_(cuda_f32(T))
    H.call("hyrf_composite_background", r._bg_args(), r.ws["b"])
    torch.cuda.synchronize()
    C, cs = oracle.background(cam, w.fields, w.bg, Cfg, T)
    assert np.abs(np_(r.C) - C).max() < TOL_IMG_F32
    dC = rng.standard_normal((70, 90, 3)).astype(np.float32)
    r.dC.copy_(cuda_f32(dC))
    m.zero_grad()
    H.hyrf_composite_background_backward(r._bg_args(), ws=r.ws["bb"], d_C=r.dC, d_C_fg=None,
                                         d_T_final=r.dT, grads=m.grads_struct(), loss_scale=1.0)
    torch.cuda.synchronize()
    g = oracle.background_backward(cam, w.fields, w.bg, T, dC)
    assert rel_l2(np_(r.dT), g["T_final"]) < TOL_GRAD_F32
    assert rel_l2(np_(m.grad["rad_table"]), g["rad_table"]) < TOL_GRAD_F32
    for l in range(2):
        assert rel_l2(np_(m.grad["col_W"][l]), g["col_W"][l]) < TOL_GRAD_F32
        assert rel_l2(np_(m.grad["col_b"][l]), g["col_b"][l]) < TOL_GRAD_F32


@pytest.mark.parametrize("lam", [0.0, 0.2])
def test_loss_matches_oracle(lib, lam):
    rng = np.random.default_rng(8)
    Hh, W = 61, 83
    x = rng.uniform(0, 1, (Hh, W, 3)).astype(np.float32)
    y = rng.uniform(0, 1, (Hh, W, 3)).astype(np.float32)
    dev = "cuda"
    loss = torch.zeros(1, device=dev)
    dC = torch.zeros(Hh, W, 3, device=dev)
    H.hyrf_loss(width=W, height=Hh, C=cuda_f32(x), target=cuda_f32(y), lam=lam, grad_scale=1.0,
                loss=loss, d_C=dC)
    torch.cuda.synchronize()
    L, g = oracle.loss(x, y, lam)
    assert abs(float(loss.item()) - L) < 1e-5 * max(1, abs(L))
    assert rel_l2(np_(dC), g) < TOL_GRAD_F32


# ------------------------------------------------------------------ kernel timer

def test_kernel_timer_counts_each_launch(lib):
    w = _cfg("c1")
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg)
    r.forward()
    torch.cuda.synchronize()
    H.hyrf_timer_read()                      # clear
    H.hyrf_timer_enable(True)
    l0 = H.launch_count()
    try:
        r.forward()
    finally:
        H.hyrf_timer_enable(False)
    launched = H.launch_count() - l0
    t = H.hyrf_timer_read()
    assert sum(n for n, _ in t.values()) == launched
    assert t["k_raster_fwd"][0] == 1 and t["k_project"][0] == 1
    assert all(ms >= 0.0 for _, ms in t.values())
    assert H.hyrf_timer_read() == {}         # totals were cleared
    r.forward()                              # disabled: nothing recorded
    torch.cuda.synchronize()
    assert H.hyrf_timer_read() == {}


# ------------------------------------------------------------------ storage order

def test_spatial_order_is_a_locality_preserving_permutation(lib):
    w = synth.config3(n=200_000, width=320, height=240, log2_T=14, n_clusters=64, precision="f32")
    m = DeviceModel(w)
    before = np_(m.pos).copy()
    cols = {k: np_(getattr(m, k)).copy() for k in ("alpha_e", "scale_e", "color_e")}
    perm = np_(m.spatial_order())
    torch.cuda.synchronize()
    n = len(before)
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.array_equal(np_(m.pos), before[perm])
    for k, v in cols.items():
        assert np.array_equal(np_(getattr(m, k)), v[perm]), k
    step_new = np.linalg.norm(np.diff(np_(m.pos), axis=0), axis=1).mean()
    step_old = np.linalg.norm(np.diff(before, axis=0), axis=1).mean()
    assert step_new < 0.1 * step_old, (step_new, step_old)


def test_bounded_wait_gives_up_with_a_status():
    """The tensor-core kernels' bounded wait, on a barrier that nothing
    completes: the kernel gives up after its polls, reports
    HYRF_ERR_TIMEOUT in the status word and the context stays usable."""
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    H.hyrf_check_bounded_wait(st, 1000)
    assert H.read_status(st) & H.HYRF_ERR_TIMEOUT
    st.zero_()
    torch.cuda.synchronize()  # the context still works
    assert H.read_status(st) == 0
    with pytest.raises(H.HyrfError):
        H.hyrf_check_bounded_wait(st, 0)


def test_bounded_wait_time_per_poll():
    """Wall time of one poll of the bounded wait (mbarrier.try_wait, which may
    suspend the thread for a hardware-chosen time), from CUDA events around
    waits of 2^14 and 2^16 polls: the tensor-core kernels give up after 2^20
    polls, so a wait that never completes ends after 2^20 times this."""
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    H.hyrf_check_bounded_wait(st, 16)  # load the kernel
    torch.cuda.synchronize()
    ms = {}
    for polls in (1 << 14, 1 << 16):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        H.hyrf_check_bounded_wait(st, polls)
        e1.record()
        torch.cuda.synchronize()
        ms[polls] = e0.elapsed_time(e1)
    assert H.read_status(st) & H.HYRF_ERR_TIMEOUT
    per_poll_us = (ms[1 << 16] - ms[1 << 14]) * 1e3 / ((1 << 16) - (1 << 14))
    print(f"bounded wait: {per_poll_us * 1e3:.1f} ns per poll; 2^20 polls = {per_poll_us * (1 << 20) / 1e6:.2f} s")
    assert per_poll_us > 0
