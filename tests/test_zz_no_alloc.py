"""hyrf_bin_sort_noalloc: the bin/sort stage for callers that cannot
allocate device memory. It must give exactly what hyrf_bin_sort gives (keys,
instance list, tile ranges and instance count are integers: bit-exact), on
two calls in a row (the shared scratch array keeps the previous call's
contents), and must refuse sizes beyond its fixed scratch array. This file
is collected last on purpose."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_17083_gb300 import hyrf as H
from paper_2509_17083_gb300 import synth

pytestmark = pytest.mark.gpu


def _inputs(seed, n, W, Hh):
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(-2.5, 2.5, n), rng.uniform(-1.6, 1.6, n), rng.uniform(1.0, 8.0, n)], 1)
    s = np.exp(rng.uniform(-5, -2, (n, 3)))
    q = synth.random_quats(rng, n)
    cam = synth.pinhole(W, Hh, 60.0)
    rect, ntiles, depth, _ = oracle.project_f32(pos.astype(np.float32), s.astype(np.float32),
                                                q.astype(np.float32), cam)
    depth[: n // 8] = depth[n // 8: 2 * (n // 8)]  # equal keys
    return rect, ntiles, depth, oracle.tiles_of(W, Hh)


def _outputs(n, cap, ntiles_total_tiles):
    d = "cuda"
    return dict(keys=torch.full((cap,), -1, dtype=torch.int64, device=d),
                vals=torch.full((cap,), -1, dtype=torch.int32, device=d),
                ranges=torch.full((ntiles_total_tiles, 2), -1, dtype=torch.int32, device=d),
                n_instances=torch.zeros(1, dtype=torch.int32, device=d),
                status=torch.zeros(1, dtype=torch.int32, device=d))


def _args(rect, ntiles, depth, TX, TY, n, cap):
    d = "cuda"
    return dict(n=n, n_vis=torch.tensor([n], dtype=torch.int32, device=d),
                rect=torch.as_tensor(rect).to(d), ntiles=torch.as_tensor(ntiles).to(d),
                depth=torch.as_tensor(depth).to(d), tiles_x=TX, tiles_y=TY, capacity=cap)


def test_noalloc_matches_workspace_version_twice():
    cases = [(1, 20000, 333, 211), (2, 3000, 129, 97)]  # second call: smaller, different sizes
    for seed, n, W, Hh in cases:
        rect, ntiles, depth, (TX, TY) = _inputs(seed, n, W, Hh)
        K = int(ntiles.sum())
        cap = K + 17
        assert n <= H.NOALLOC_MAX_GAUSSIANS and cap <= H.NOALLOC_MAX_INSTANCES
        args = _args(rect, ntiles, depth, TX, TY, n, cap)
        ref = _outputs(n, cap, TX * TY)
        H.hyrf_bin_sort(**args, **ref)
        got = _outputs(n, cap, TX * TY)
        H.hyrf_bin_sort_noalloc(**args, **got)
        torch.cuda.synchronize()
        assert int(got["n_instances"].item()) == int(ref["n_instances"].item()) == K
        for key in ("keys", "vals", "ranges"):
            a, b = ref[key].cpu().numpy(), got[key].cpu().numpy()
            if key != "ranges":
                a, b = a[:K], b[:K]
            assert np.array_equal(a, b), key
        assert H.read_status(got["status"]) == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    rect, ntiles, depth, (TX, TY) = _inputs(3, 100, 64, 48)
    args = _args(rect, ntiles, depth, TX, TY, 100, int(ntiles.sum()))
    args["capacity"] = H.NOALLOC_MAX_INSTANCES + 1
    with pytest.raises(H.HyrfError):
        H.hyrf_bin_sort_noalloc(**args, **_outputs(100, 16, TX * TY))
    args["capacity"] = 1000
    args["n"] = H.NOALLOC_MAX_GAUSSIANS + 1
    with pytest.raises(H.HyrfError):
        H.hyrf_bin_sort_noalloc(**args, **_outputs(100, 16, TX * TY))
