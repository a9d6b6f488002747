"""Run a few training iterations (or render-only forwards) of one workload,
for external profilers: every library call of the step is issued from the
host (no CUDA graph), so a profiler sees each launch with its name.

  python -m paper_2509_17083_gb300.step_driver [--config 3] [--n 1000000]
         [--precision bf16|f32] [--steps 3] [--render]

Prints the device status and the loss of the last step.
"""
import argparse

import torch

from . import hyrf as H
from . import synth
from .pipeline import DeviceModel, ViewRenderer


def workload(config, n, precision):
    if config == 1:
        return synth.config1()
    if config == 2:
        return synth.config2()
    if config == 5:
        return synth.config5()
    return synth.config3(n=n, precision=precision)


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--config", type=int, default=3, choices=[1, 2, 3, 5])
    p.add_argument("--n", type=int, default=1_000_000)
    p.add_argument("--precision", default="bf16", choices=["bf16", "f32"])
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--render", action="store_true", help="forward only")
    a = p.parse_args(argv)
    if not torch.cuda.is_available():
        raise SystemExit("needs a CUDA GPU")
    w = workload(a.config, a.n, a.precision)
    m = DeviceModel(w)
    m.spatial_order()
    r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
    tgt = torch.as_tensor(w.targets[0]).cuda()
    r.fit_capacity(tgt)
    for _ in range(a.steps):
        if a.render:
            r.forward(None, want_keys=False)
        else:
            m.zero_grad()
            r.step(tgt)
    torch.cuda.synchronize()
    print(f"status {H.read_status(r.status)} loss {float(r.loss.item()):.6f} "
          f"visible {int(r.n_vis.item())} instances {int(r.n_inst.item())}")


if __name__ == "__main__":
    main()
