"""Fused multi-tensor Adam on the GPU against the FP64 oracle's Adam, over
ragged tensor sizes (vector body and scalar tail), several steps, and the
bf16 working copy of a master tensor."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_17083_gb300 import hyrf as H
from tests.gpu_util import np_

pytestmark = pytest.mark.gpu


def test_adam_matches_oracle_over_ragged_tensors():
    rng = np.random.default_rng(41)
    sizes = [1, 3, 4096, 4097, 123457, 1 << 20]
    dev = "cuda"
    ts, ref = [], []
    for i, n in enumerate(sizes):
        p = rng.standard_normal(n).astype(np.float32)
        t = dict(param=torch.tensor(p, device=dev), grad=torch.zeros(n, device=dev),
                 m=torch.zeros(n, device=dev), v=torch.zeros(n, device=dev),
                 lr_scale=float(0.5 + i))
        if i % 2:
            t["shadow"] = torch.zeros(n, dtype=torch.bfloat16, device=dev)
        ts.append(t)
        ref.append([p.astype(np.float64), np.zeros(n), np.zeros(n)])
    # the hyper-parameters cross the C ABI as float32: the oracle takes the
    # same float32 values (0.999 as float32 is 0.99900001287...)
    lr, b1, b2, eps, gs = [float(np.float32(x)) for x in (1e-3, 0.9, 0.999, 1e-8, 0.5)]
    for step in range(1, 4):
        for t, r in zip(ts, ref):
            g = (rng.standard_normal(t["param"].numel()) * 1e-2).astype(np.float32)
            t["grad"].copy_(torch.tensor(g, device=dev))
            lrt = float(np.float32(lr) * np.float32(t["lr_scale"]))
            r[0], r[1], r[2] = oracle.adam_step(r[0], g, r[1], r[2], lrt, b1, b2, eps, step, grad_scale=gs)
        H.hyrf_adam_step(ts, lr, b1, b2, eps, step, grad_scale=gs)
        torch.cuda.synchronize()
    for t, r in zip(ts, ref):
        p = np_(t["param"])
        np.testing.assert_allclose(p, r[0], rtol=1e-6, atol=2e-6)
        np.testing.assert_allclose(np_(t["m"]), r[1], rtol=1e-5, atol=1e-9)
        np.testing.assert_allclose(np_(t["v"]), r[2], rtol=1e-5, atol=1e-12)
        if "shadow" in t:
            assert torch.equal(t["shadow"], t["param"].to(torch.bfloat16))


def test_adam_rejects_bad_arguments():
    x = torch.zeros(8, device="cuda")
    with pytest.raises(H.HyrfError):
        H.hyrf_adam_step([dict(param=x, grad=x, m=x, v=x)], 1e-3, 0.9, 0.999, 1e-8, step=0)
    with pytest.raises(H.HyrfError):
        H.hyrf_adam_step([dict(param=x, grad=x, m=x, v=x)], 1e-3, 1.0, 0.999, 1e-8, step=1)
