"""End-to-end pins of the composed oracle path (Fig. 3 pipeline, Eq. 12).

(1) With the decoders reduced to their biases (so the background is a
constant 0.5), HyRF degenerates to plain isotropic 3DGS (the "w/o Neural" case of
Tab. 5); that case is checked against a brute-force per-pixel splat written
from the 3DGS definition for isotropic Gaussians.
(2) The analytic gradient of the loss with respect to every parameter class
matches central finite differences of the forward pass.
"""
import numpy as np
import pytest

import oracle
from paper_2509_17083_gb300 import synth

sig = lambda x: 1.0 / (1.0 + np.exp(-x))


def test_reduces_to_isotropic_3dgs(orc):
    w = synth.config1(n=60, width=48, height=40, table_init=0.3, seed=3)
    fl = w.fields
    for m in (fl.geo_mlp, fl.col_mlp):
        m.W = [np.zeros_like(x) for x in m.W]
    # zero decoders: the background colour is sigma(0) = 0.5 everywhere
    g = w.gaussians
    cam = w.cams[0]
    fw = oracle.render(g, fl, cam, w.bg)
    ids = fw["ids"]
    a = sig(g.alpha_e[ids].astype(np.float64))
    s = sig(g.scale_e[ids].astype(np.float64))
    col = sig(g.color_e[ids].astype(np.float64))
    p = g.pos[ids].astype(np.float64)
    # brute force: per pixel, all Gaussians in the pixel's tile, by depth
    TX = (cam.width + 15) // 16
    order = np.argsort(fw["depth32"], kind="stable")
    img = np.zeros((cam.height, cam.width, 3))
    for py in range(cam.height):
        for px in range(cam.width):
            T = 1.0
            for k in order:
                r = fw["rect"][k]
                if not (r[0] <= px // 16 < r[2] and r[1] <= py // 16 < r[3]):
                    continue
                x, y, z = p[k]
                J = np.array([[cam.fx / z, 0, -cam.fx * x / z ** 2], [0, cam.fy / z, -cam.fy * y / z ** 2]])
                S = s[k] ** 2 * J @ J.T + 0.3 * np.eye(2)
                d = np.array([cam.fx * x / z + cam.cx - px - 0.5, cam.fy * y / z + cam.cy - py - 0.5])
                al = min(0.99, a[k] * np.exp(-0.5 * d @ np.linalg.solve(S, d)))
                if al < 1 / 255:
                    continue
                if T * (1 - al) < 1e-4:
                    break
                img[py, px] += col[k] * al * T
                T *= 1 - al
            img[py, px] += 0.5 * T
    np.testing.assert_allclose(fw["C"], img, atol=1e-12)


def _fd_check(w, rng, n_per_class=6, h_rel=1e-6, rtol=2e-4):
    g, fl, cam, bg, tgt, lam = w.gaussians, w.fields, w.cams[0], w.bg, w.targets[0], w.ssim_lambda
    # float64 copies so that +-h is representable
    g.pos, g.alpha_e, g.scale_e, g.color_e = [np.asarray(x, np.float64) for x in
                                              (g.pos, g.alpha_e, g.scale_e, g.color_e)]
    for grid in (fl.geo, fl.rad):
        grid.table = grid.table.astype(np.float64)
    for m in (fl.geo_mlp, fl.col_mlp):
        m.W = [x.astype(np.float64) for x in m.W]
        m.b = [x.astype(np.float64) for x in m.b]
    L0, fw0, grads, _ = oracle.loss_and_grads(g, fl, cam, bg, tgt, lam)

    def sig_of(fw):
        return (fw["vis"].tobytes(), fw["rect"].tobytes(), fw["vals"].tobytes(),
                fw["n_contrib"].tobytes(), np.sign(fw["C"] - tgt).tobytes())

    base = sig_of(fw0)

    def fd(arr, e):
        v = arr[e]
        h = h_rel * max(1.0, abs(v))
        arr[e] = v + h
        fp = oracle.render(g, fl, cam, bg)
        lp = oracle.loss(fp["C"], tgt, lam)[0]
        arr[e] = v - h
        fm = oracle.render(g, fl, cam, bg)
        lm = oracle.loss(fm["C"], tgt, lam)[0]
        arr[e] = v
        if sig_of(fp) != base or sig_of(fm) != base:
            return None  # a discrete decision moved: not differentiable here
        if min(fp["margin"].min(), fm["margin"].min()) < 1e-6:
            return None
        return (lp - lm) / (2 * h)

    checked = {}
    vis_ids = fw0["ids"]
    classes = [("pos", g.pos, lambda: (rng.choice(vis_ids), rng.integers(3))),
               ("alpha_e", g.alpha_e, lambda: (rng.choice(vis_ids),)),
               ("scale_e", g.scale_e, lambda: (rng.choice(vis_ids),)),
               ("color_e", g.color_e, lambda: (rng.choice(vis_ids), rng.integers(3)))]
    for key, grid in [("geo_table", fl.geo.table), ("rad_table", fl.rad.table)]:
        nz = np.argwhere(np.abs(grads[key]) > 1e-9)
        classes.append((key, grid, lambda nz=nz: tuple(nz[rng.integers(len(nz))])))
    for key, m in [("geo", fl.geo_mlp), ("col", fl.col_mlp)]:
        for l in range(m.n_hidden + 1):
            W = m.W[l]
            classes.append((f"{key}_W{l}", W, lambda W=W: (rng.integers(W.shape[0]), rng.integers(W.shape[1]))))
    for key, arr, pick in classes:
        ok = 0
        for _ in range(n_per_class * 4):
            e = pick()
            num = fd(arr, e)
            if num is None:
                continue
            if key.startswith(("geo_W", "col_W")):
                l = int(key[-1])
                ana = grads[key[:-1]][l][e]
            else:
                ana = grads[key][e]
            np.testing.assert_allclose(ana, num, rtol=rtol, atol=1e-9 + 1e-6 * abs(L0),
                                       err_msg=f"{key}{e}")
            ok += 1
            if ok == n_per_class:
                break
        checked[key] = ok
        assert ok >= n_per_class // 2, (key, ok)
    return checked


def test_end_to_end_gradient_map_background_l1(orc):
    w = synth.config1(n=150, width=40, height=32, table_init=0.5, seed=1)
    w.bg = synth.Background(1, 6, 10)
    _fd_check(w, np.random.default_rng(0))


def test_end_to_end_gradient_exact_background_ssim(orc):
    w = synth.config1(n=120, width=36, height=28, table_init=0.5, seed=2)
    w.bg = synth.Background(0)
    w.ssim_lambda = 0.2
    _fd_check(w, np.random.default_rng(1))
