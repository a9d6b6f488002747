"""Training iterations with the fused Adam update toward a teacher-rendered
target: the student (the scene with its own explicit colours and opacities)
learns the teacher's image (the same scene with other explicit colours and
opacities). BF16 and FP32 fields must both converge, to PSNRs that agree.
"""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2509_17083_gb300 import hyrf as H
from paper_2509_17083_gb300 import synth
from paper_2509_17083_gb300.pipeline import DeviceModel, Trainer, ViewRenderer

pytestmark = pytest.mark.gpu


def _psnr(a, b):
    return float(-10.0 * torch.log10(((a.clamp(0, 1) - b) ** 2).mean()))


def _train(precision, steps=60):
    w = synth.config3(n=30000, width=301, height=203, log2_T=15, n_clusters=32, precision=precision)
    rng = np.random.default_rng(51)
    g = w.gaussians
    teacher = dataclasses.replace(w, gaussians=dataclasses.replace(
        g, color_e=rng.standard_normal(g.color_e.shape).astype(np.float32),
        alpha_e=(g.alpha_e + 1.0).astype(np.float32)))
    tm = DeviceModel(teacher)
    tr = ViewRenderer(tm, w.cams[0], w.bg)
    tr.fit_capacity()
    target = tr.forward(None).clone()
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
    r.fit_capacity(target)
    tr_ = Trainer(m, [r])
    losses = []
    p0 = None
    for k in range(steps):
        r.status.zero_()
        loss = tr_.step([target])[0]
        losses.append(float(loss.item()))
        if k == 0:
            p0 = _psnr(r.C, target)
        assert H.read_status(r.status) == 0
    r.forward(None)
    torch.cuda.synchronize()
    return losses, p0, _psnr(r.C, target)


@pytest.fixture(scope="module")
def runs():
    return {p: _train(p) for p in ("bf16", "f32")}


@pytest.mark.parametrize("precision", ["bf16", "f32"])
def test_training_converges_toward_teacher(runs, precision):
    losses, p0, p1 = runs[precision]
    assert losses[-1] < 0.6 * losses[0], (losses[0], losses[-1])
    assert p1 > p0 + 3.0, (p0, p1)


def test_bf16_and_fp32_training_agree(runs):
    _, _, pb = runs["bf16"]
    _, _, pf = runs["f32"]
    assert abs(pb - pf) < 0.5, (pb, pf)


def test_training_with_density_control():
    """Densify (clone / split), prune and reset opacity during training: the
    Gaussian count changes, every buffer is rebuilt consistently and the loss
    keeps falling."""
    w = synth.config3(n=30000, width=301, height=203, log2_T=15, n_clusters=32, precision="bf16")
    rng = np.random.default_rng(52)
    g = w.gaussians
    teacher = dataclasses.replace(w, gaussians=dataclasses.replace(
        g, color_e=rng.standard_normal(g.color_e.shape).astype(np.float32)))
    tm = DeviceModel(teacher)
    tr = ViewRenderer(tm, w.cams[0], w.bg)
    tr.fit_capacity()
    target = tr.forward(None).clone()
    m = DeviceModel(w)
    r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
    r.fit_capacity(target)
    trainer = Trainer(m, [r])
    losses, counts = [], [m.n]
    for k in range(1, 61):
        losses.append(float(trainer.step([target])[0].item()))
        assert H.read_status(trainer.views[0].status) == 0
        if k % 15 == 0:
            counts.append(trainer.densify([target], grad_threshold=2e-6))
            assert trainer.m.n == counts[-1] and trainer.m.pos.shape[0] == counts[-1]
        if k == 30:
            trainer.reset_opacity()
    assert counts[1] != counts[0], counts
    assert max(counts) > counts[0], counts  # some Gaussians were cloned or split
    assert np.mean(losses[-5:]) < 0.8 * np.mean(losses[:5]), (losses[:5], losses[-5:])
