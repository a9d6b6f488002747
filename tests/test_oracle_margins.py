"""Pins of the oracle helpers that decide which pixels and rows the parity
tests compare, and of the decoders' BF16 ReLU-branch replay.

* The replay (orc_mlp.relu_replay = 1) on hand-built decoders whose branch
  flips when the layer input, or the hidden output, is rounded to bfloat16
  (8 significand bits: the neighbours of 1 are 1 - 2^-8 and 1 + 2^-7).
* decoder_margins / bg_margins / relu_safe_mask on hand-built decoders fed by
  constant grids (every feature equals the table value, Eq. 3 interpolates a
  constant exactly), whose pre-activations are known numbers.
* decision_safe_mask: the compositing-threshold part on one isotropic
  Gaussian (closed form of Eq. 1's alpha), and the tile-rectangle part on a
  Gaussian whose 3-sigma radius sits exactly on an integer (the ceil of the
  3DGS radius flips under the mask's perturbation).
"""
import dataclasses

import numpy as np
import pytest

from paper_2509_17083_gb300 import synth


def _mlp(Ws, bs):
    Ws = [np.asarray(w, np.float64) for w in Ws]
    bs = [np.asarray(b, np.float64) for b in bs]
    return synth.MLP(n_in=Ws[0].shape[1], width=Ws[0].shape[0], n_hidden=len(Ws) - 1,
                     n_out=Ws[-1].shape[0], W=Ws, b=bs)


def test_relu_replay_rounds_layer_inputs(orc):
    # x0 = 1 + 2^-10 rounds to 1 in bfloat16: the FP64 pre-activation of unit 0
    # is +2^-11, the replay's is -2^-11 (branch off); unit 1 is far from its kink
    m = _mlp([[[1.0, 0.0], [0.0, 1.0]], [[1.0, 1.0]]], [[-(1 + 2.0 ** -11), 0.25], [0.0]])
    x = [1 + 2.0 ** -10, 0.0]
    assert orc.mlp_forward(m, x, relu="f64")[0] == 0.25 + 2.0 ** -11
    assert orc.mlp_forward(m, x, relu="bf16")[0] == 0.25
    # an input that bfloat16 represents exactly takes the same branch both ways
    x = [1 + 2.0 ** -7, 0.0]
    assert orc.mlp_forward(m, x, relu="bf16")[0] == orc.mlp_forward(m, x, relu="f64")[0]


def test_branch_sum_tracks_branch_patterns(orc):
    m = _mlp([[[1.0, 0.0], [0.0, 1.0]], [[1.0, 1.0]]], [[-(1 + 2.0 ** -11), 0.25], [0.0]])
    sums = []
    for x, relu in [([1 + 2.0 ** -10, 0.0], "f64"), ([1 + 2.0 ** -10, 0.0], "f64"),
                    ([1 + 2.0 ** -10, 0.0], "bf16"), ([2.0, 0.0], "f64"), ([2.0, 0.0], "bf16")]:
        orc.branch_sum_reset()
        orc.mlp_forward(m, x, relu=relu)
        sums.append(orc.branch_sum())
    # same pattern, same sum; unit 0 off in the replay; both on for x0 = 2
    assert sums[0] == sums[1] == sums[3] == sums[4] != sums[2]
    orc.branch_sum_reset()
    orc.mlp_forward(m, [2.0, 0.0])
    orc.mlp_forward(m, [2.0, 0.0], relu="bf16")
    assert orc.branch_sum() == (2 * sums[0]) % 2 ** 64


def test_relu_replay_rounds_hidden_outputs(orc):
    # layer 0 passes z = 1 + 2^-9 (FP64); bfloat16 rounds it to 1, so layer
    # 1's pre-activation is 2^-10 in FP64 and -2^-10 in the replay
    m = _mlp([[[1.0]], [[1.0]], [[1.0]]], [[2.0 ** -9], [-(1 + 2.0 ** -10)], [0.5]])
    x = [1.0]
    assert orc.mlp_forward(m, x, relu="f64")[0] == 0.5 + 2.0 ** -10
    assert orc.mlp_forward(m, x, relu="bf16")[0] == 0.5


def _const_fields(c=0.5):
    """Constant 2-level grids (features all c) and hand-built decoders:
    geometry hidden pre-activations (c - c + 0.01, c/2 - 0.2) = (0.01, 0.05)
    with magnitudes (c + c + 0.01, c/2 + 0.2) -> margin min(0.01/1.01,
    0.05/0.45) = 0.01/1.01; colour (c - 0.45, 0.3) = (0.05, 0.3), magnitudes
    (c + 0.45, 0.3) -> margin 0.05/0.95 (PE columns carry zero weight)."""
    rng = np.random.default_rng(0)
    f = synth.make_fields(rng, [-1, -1, 1], [1, 1, 3], n_levels=2, log2_T=8, width=2, n_hidden=1)
    for g in (f.geo, f.rad):
        g.table = np.full_like(g.table, c)
    Wg = np.zeros((2, 4))
    Wg[0, 0], Wg[0, 1], Wg[1, 0] = 1.0, -1.0, 0.5
    f.geo_mlp = _mlp([Wg, np.ones((8, 2))], [[0.01, -0.2], np.zeros(8)])
    Wc = np.zeros((2, 4 + f.pe_pad))
    Wc[0, 3] = 1.0
    f.col_mlp = _mlp([Wc, np.ones((3, 2))], [[-0.45, 0.3], np.zeros(3)])
    return f


def test_decoder_and_background_margins_hand_built(orc):
    f = _const_fields()
    cam = synth.pinhole(24, 16, 60.0)
    pos = np.array([[0.1, -0.2, 2.0], [0.5, 0.3, 2.5], [-0.7, 0.0, 1.4]])
    mg, mc = orc.decoder_margins(pos, cam, f)
    np.testing.assert_allclose(mg, 0.01 / 1.01, rtol=1e-12)
    np.testing.assert_allclose(mc, 0.05 / 0.95, rtol=1e-12)
    for mode in (0, 1):
        bgm = orc.bg_margins(cam, f, synth.Background(mode, 4, 8))
        assert bgm.shape == (16, 24)
        np.testing.assert_allclose(bgm, 0.05 / 0.95, rtol=1e-12)
    g = synth.Gaussians(pos=pos.astype(np.float32), alpha_e=np.zeros(3, np.float32),
                        scale_e=np.zeros(3, np.float32), color_e=np.zeros((3, 3), np.float32))
    ids = np.arange(3)
    assert orc.relu_safe_mask(g, f, cam, ids, 0.009, 0.05).tolist() == [1, 1, 1]
    assert orc.relu_safe_mask(g, f, cam, ids, 0.0100, 0.05).tolist() == [0, 0, 0]
    assert orc.relu_safe_mask(g, f, cam, ids, 0.009, 0.0527).tolist() == [0, 0, 0]
    # the replay measures the same margins here (c, 0.01, -0.2, ... are
    # bfloat16-representable apart from the biases, which stay FP64)
    mg_r, mc_r = orc.decoder_margins(pos, cam, orc.replay_relu(f, "bf16"))
    np.testing.assert_allclose(mg_r, mg, rtol=1e-12)
    np.testing.assert_allclose(mc_r, mc, rtol=1e-12)


def _fw(cam, mean, conic, margin=None):
    return dict(margin=np.ones((cam.height, cam.width)) if margin is None else margin,
                mean2d=np.asarray(mean, np.float64).reshape(-1, 2),
                conic=np.asarray(conic, np.float64).reshape(-1, 3))


def test_decision_safe_mask_tile_edges(orc):
    """One Gaussian at (40.5, 40.5) with Sigma' = diag(64/9, 64/9): 3 sqrt(lambda)
    = 8 exactly, so the radius ceil(8 (1 +- 1e-5)) is 8 or 9 and the rectangle
    [2,4)x[2,4) grows to [1,4)x[1,4) in tiles: the L-shaped difference is
    unsafe, everything else safe."""
    cam = synth.pinhole(96, 80, 60.0)
    mask = orc.decision_safe_mask(_fw(cam, [40.5, 40.5], [9 / 64, 0, 9 / 64]), cam)
    bad = np.zeros((5, 6), bool)
    bad[1:4, 1] = True
    bad[1, 1:4] = True
    np.testing.assert_array_equal(mask, ~np.kron(bad, np.ones((16, 16), bool)))
    # a radius of 7.5 (3 sqrt(lambda) = 7.5 -> ceil 8 either way) leaves every tile safe
    assert orc.decision_safe_mask(_fw(cam, [40.5, 40.5], [0.16, 0, 0.16]), cam).all()


def test_decision_safe_mask_compositing_thresholds(orc):
    """One isotropic Gaussian at a pixel centre, conic (1/v, 0, 1/v), opacity o
    chosen so that at distance^2 = 25 alpha = o exp(-25 / (2 v)) lies 5e-5
    (relative) above 1/255: those 12 pixels (3-4-5 and 5-0 offsets) are
    unsafe at the default 1e-4 margin, safe at 1e-5."""
    cam = synth.pinhole(48, 48, 60.0)
    v = 20.0
    o = (1 + 5e-5) / 255 * np.exp(25 / (2 * v))
    C, T, nc, mg = orc.rasterize(48, 48, np.array([[0, 1], [0, 1], [0, 1], [0, 1], [0, 1], [0, 1],
                                                    [0, 1], [0, 1], [0, 1]], np.int32),
                                 np.array([0], np.int32), np.array([[24.5, 24.5]]),
                                 np.array([[1 / v, 0, 1 / v]]), np.array([o]), np.array([[1.0, 0, 0]]))
    yy, xx = np.mgrid[0:48, 0:48]
    d2 = (xx - 24) ** 2 + (yy - 24) ** 2
    near = d2 == 25
    assert near.sum() == 12
    fw = _fw(cam, [24.5, 24.5], [1 / v, 0, 1 / v], margin=mg)
    # a wide Gaussian: its rectangle covers the whole 3x3-tile image whatever the perturbation
    m = orc.decision_safe_mask(fw, cam)
    np.testing.assert_array_equal(m, ~near)
    assert orc.decision_safe_mask(fw, cam, comp_margin=1e-5).all()
    # Eq. 1 closed form at the same pixels: alpha above 1/255 by 5e-5 relative
    np.testing.assert_allclose(C[near][:, 0], (1 + 5e-5) / 255, rtol=1e-12)


def test_replay_fields_copy_is_shallow_and_tagged(orc):
    f = _const_fields()
    r = orc.replay_relu(f, "bf16")
    assert r.relu_precision == "bf16" and not hasattr(f, "relu_precision")
    assert r.geo is f.geo and dataclasses.is_dataclass(r)
    with pytest.raises(ValueError):
        orc.replay_relu(f, "f16")
