"""Central finite differences of the FP64 oracle's loss against the BF16
path's analytic gradient on the headline workload: 1M Gaussians (256
clusters + 10 % far points), 16-level 2^19 bfloat16 grids, 32->64->64
decoders, exact background, L1 loss (Sec. 3.1 Eq. 1, Sec. 3.2 Eqs. 2-7,
Sec. 3.3 Eqs. 10-12).

The view is a 96x64 window of the 1237x822 camera (its principal point
shifted), so that the oracle renders it in a fraction of a second: every
Gaussian of the scene goes through the pre-cull, the window's visible ones
through every stage. 64 parameters are sampled, 16 in each class:
per-Gaussian (position, explicit opacity, scale and colour logits), table
entries reached by the window's Gaussians, decoder weights, and radiance
table entries reached by the window's background rays. Each derivative is
(L(theta + h) - L(theta - h)) / 2h with h = 1e-6 max(1, |theta|) in FP64
(table and weight entries drawn among those whose gradient is at least
1e-3 of their class's largest); a
sample is rejected (and another drawn) where the perturbation moves a
discrete decision: visibility, a tile rectangle, the instance list, a
pixel's last contributor, the sign of an L1 residual, a compositing
threshold within 1e-6 (relative), or any decoder's ReLU branch. The oracle
takes the decoders' ReLU branches as the BF16 kernels take them
(oracle.replay_relu: a replayed branch that flips makes the FP64 values
jump, so such steps must be rejected, not averaged), and Gaussians
whose replayed pre-activations are within RELU_REPLAY_MARGIN_BF16 of a kink
are not sampled. Each class must agree within the BF16 gradient tolerance
(2e-2 relative L2 over its 16 samples).
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2509_17083_gb300 import hyrf as H
from paper_2509_17083_gb300 import synth
from paper_2509_17083_gb300.pipeline import DeviceModel, ViewRenderer
from tests.gpu_util import RELU_REPLAY_MARGIN_BF16, TOL_GRAD_BF16, cuda_f32, np_, rel_l2

pytestmark = pytest.mark.gpu

CW, CH = 96, 64
PER_CLASS = 16


def _window(cam, x0, y0):
    return dataclasses.replace(cam, cx=cam.cx - x0, cy=cam.cy - y0, width=CW, height=CH)


def _pick_window(w, rng):
    """First seeded window whose pre-cull keeps 3,000-6,000 Gaussians."""
    cam = w.cams[0]
    for _ in range(200):
        x0 = int(rng.integers(0, cam.width - CW))
        y0 = int(rng.integers(0, cam.height - CH))
        nv = int(oracle.precull_f32(w.gaussians.pos, _window(cam, x0, y0)).sum())
        if 3000 <= nv <= 6000:
            return x0, y0
    raise AssertionError("no window of the wanted size")


@pytest.fixture(scope="module")
def fd_case():
    w = synth.config3()
    rng = np.random.default_rng(2)
    x0, y0 = _pick_window(w, rng)
    cam = _window(w.cams[0], x0, y0)
    tgt = np.ascontiguousarray(w.targets[0][y0:y0 + CH, x0:x0 + CW])
    # GPU: one training iteration of the window through the BF16 path
    m = DeviceModel(w)
    r = ViewRenderer(m, cam, w.bg, lam=0.0, loss_scale=w.loss_scale)
    t = cuda_f32(tgt)
    r.fit_capacity(t)
    m.zero_grad()
    r.status.zero_()
    r.step(t)
    torch.cuda.synchronize()
    assert H.read_status(r.status) == 0
    gpu = {k: ([np_(x) for x in v] if isinstance(v, list) else np_(v)) for k, v in m.grad.items()}
    loss_gpu = float(r.loss.item())
    del r, m
    torch.cuda.empty_cache()
    return w, cam, tgt, gpu, loss_gpu, rng


def _f64_params(w):
    """FP64 copies of every parameter (so that theta +- h is representable);
    the values are the BF16 path's."""
    g = dataclasses.replace(w.gaussians, pos=w.gaussians.pos.astype(np.float64),
                            alpha_e=w.gaussians.alpha_e.astype(np.float64),
                            scale_e=w.gaussians.scale_e.astype(np.float64),
                            color_e=w.gaussians.color_e.astype(np.float64))
    fl = w.fields
    grids = [dataclasses.replace(x, table=x.table.astype(np.float64)) for x in (fl.geo, fl.rad)]
    mlps = [dataclasses.replace(x, W=[a.astype(np.float64) for a in x.W], b=[a.astype(np.float64) for a in x.b])
            for x in (fl.geo_mlp, fl.col_mlp)]
    f = dataclasses.replace(fl, geo=grids[0], rad=grids[1], geo_mlp=mlps[0], col_mlp=mlps[1])
    return g, oracle.replay_relu(f, "bf16")


def test_config3_gradient_matches_central_differences(fd_case):
    w, cam, tgt, gpu, loss_gpu, rng = fd_case
    g, fr = _f64_params(w)
    bg = w.bg
    L0, fw0, grads, inter = oracle.loss_and_grads(g, fr, cam, bg, tgt, 0.0)
    assert abs(loss_gpu - L0) < 2e-3 * abs(L0), (loss_gpu, L0)
    gb = oracle.background_backward(cam, fr, bg, fw0["T_final"], inter["dC"])

    def render():
        oracle.branch_sum_reset()
        f = oracle.render(g, fr, cam, bg)
        f["branches"] = oracle.branch_sum()
        return f

    def sig(fw):
        return (fw["vis"].tobytes(), fw["rect"].tobytes(), fw["vals"].tobytes(),
                fw["n_contrib"].tobytes(), np.sign(fw["C"] - tgt).tobytes(), fw["branches"])

    base = sig(render())

    sign0 = np.sign(fw0["C"] - tgt)

    def fd(arr, e):
        """Central difference of the L1 loss. With no residual changing sign
        (checked), L(+h) - L(-h) = mean(sign(C - target) (C(+h) - C(-h))):
        summing the per-pixel differences keeps the rounding of the two
        ~0.3-sized losses out of derivatives as small as 1e-11 (the
        background's, behind T_final ~ 1e-4)."""
        v = arr[e]
        h = 1e-6 * max(1.0, abs(v))
        img = []
        for s in (1.0, -1.0):
            arr[e] = v + s * h
            f = render()
            if sig(f) != base or f["margin"].min() < 1e-6:
                arr[e] = v
                return None
            img.append(f["C"])
        arr[e] = v
        return float(np.sum(sign0 * (img[0] - img[1]))) / (sign0.size * 2 * h)

    ids = fw0["ids"]
    safe = oracle.relu_safe_mask(g, fr, cam, ids, RELU_REPLAY_MARGIN_BF16, RELU_REPLAY_MARGIN_BF16) > 0
    # most of the window's Gaussians are hidden behind the first few dozen
    # of each pixel (no gradient): sample the ones that move the loss
    moving = np.linalg.norm(grads["pos"][ids], axis=1) > 0
    rows = ids[safe & moving]
    assert len(rows) > max(100, 0.8 * moving.sum()), (len(rows), moving.sum())
    q_rad = grads["rad_table"] - gb["rad_table"]

    def nz(a):
        """Entries whose gradient is at least 1e-3 of the largest one."""
        return np.argwhere(np.abs(a) >= 1e-3 * np.abs(a).max())

    gaussian_kinds = [("pos", g.pos, 3), ("alpha_e", g.alpha_e, 0), ("scale_e", g.scale_e, 0),
                      ("color_e", g.color_e, 3)]

    def pick_gaussian():
        key, arr, width = gaussian_kinds[rng.integers(4)]
        i = int(rng.choice(rows))
        return key, arr, ((i, int(rng.integers(width))) if width else (i,))

    tab = {"geo_table": nz(grads["geo_table"]), "rad_table": nz(q_rad)}

    def pick_table():
        key = ("geo_table", "rad_table")[rng.integers(2)]
        e = tab[key][rng.integers(len(tab[key]))]
        return key, (fr.geo if key == "geo_table" else fr.rad).table, tuple(e)

    bg_e = nz(gb["rad_table"])

    def pick_bg():
        return "rad_table", fr.rad.table, tuple(bg_e[rng.integers(len(bg_e))])

    def pick_weight():
        name = ("geo", "col")[rng.integers(2)]
        mlp = fr.geo_mlp if name == "geo" else fr.col_mlp
        l = int(rng.integers(3))
        cand = nz(grads[f"{name}_W"][l])
        e = tuple(cand[rng.integers(len(cand))])
        return (f"{name}_W", l), mlp.W[l], e

    def gpu_value(key, e):
        if isinstance(key, tuple):
            return gpu[key[0]][key[1]][e]
        return gpu[key][e]

    def ana_value(key, e):
        if isinstance(key, tuple):
            return grads[key[0]][key[1]][e]
        return grads[key][e]

    report = {}
    for cls, pick in (("per-Gaussian", pick_gaussian), ("table entry", pick_table),
                      ("decoder weight", pick_weight), ("background", pick_bg)):
        num, got, ana = [], [], []
        for _ in range(4 * PER_CLASS):
            key, arr, e = pick()
            d = fd(arr, e)
            if d is None:
                continue
            num.append(d)
            got.append(gpu_value(key, e))
            ana.append(ana_value(key, e))
            if len(num) == PER_CLASS:
                break
        assert len(num) == PER_CLASS, (cls, len(num))
        num, got, ana = map(np.asarray, (num, got, ana))
        report[cls] = (rel_l2(got, num), rel_l2(ana, num))
    print("config-3 finite differences (GPU vs FD, oracle analytic vs FD):",
          {k: (f"{a:.2e}", f"{b:.2e}") for k, (a, b) in report.items()})
    for cls, (e_gpu, e_ana) in report.items():
        assert e_ana < 1e-4, (cls, e_ana)   # the oracle's own analytic reverse
        assert e_gpu < TOL_GRAD_BF16, (cls, e_gpu)
