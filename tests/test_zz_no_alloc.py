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


def _run_both(args, n, cap, tiles):
    ref = _outputs(n, cap, tiles)
    H.hyrf_bin_sort(**args, **ref)
    got = _outputs(n, cap, tiles)
    H.hyrf_bin_sort_noalloc(**args, **got)
    torch.cuda.synchronize()
    return ref, got


def _same(ref, got, K):
    assert int(got["n_instances"].item()) == int(ref["n_instances"].item())
    assert H.read_status(got["status"]) == H.read_status(ref["status"])
    for key in ("keys", "vals", "ranges"):
        a, b = ref[key].cpu().numpy(), got[key].cpu().numpy()
        if key != "ranges":
            a, b = a[:K], b[:K]
        assert np.array_equal(a, b), key


def test_noalloc_allocates_nothing():
    """After a first call (which looks up the scratch array's address), more
    calls leave the device's free memory and torch's allocator unchanged."""
    rect, ntiles, depth, (TX, TY) = _inputs(4, 30000, 401, 257)
    n, K = 30000, int(ntiles.sum())
    args = _args(rect, ntiles, depth, TX, TY, n, K)
    out = _outputs(n, K, TX * TY)
    H.hyrf_bin_sort_noalloc(**args, **out)
    torch.cuda.synchronize()
    free0, used0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        H.hyrf_bin_sort_noalloc(**args, **out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == used0
    assert H.read_status(out["status"]) == 0


def test_noalloc_with_depth_order_and_fewer_visible_rows():
    """The optional depth order of hyrf_depth_order, and a visible count below
    the arrays' capacity (only the first n_vis rows are binned)."""
    rng = np.random.default_rng(5)
    n, W, Hh = 12000, 321, 203
    pos = np.stack([rng.uniform(-2.5, 2.5, n), rng.uniform(-1.6, 1.6, n), rng.uniform(1.0, 8.0, n)], 1)
    s = np.exp(rng.uniform(-5, -2, (n, 3)))
    q = synth.random_quats(rng, n)
    cam = synth.pinhole(W, Hh, 60.0)
    rect, ntiles, depth, _ = oracle.project_f32(pos.astype(np.float32), s.astype(np.float32),
                                                q.astype(np.float32), cam)
    TX, TY = oracle.tiles_of(W, Hh)
    for n_vis in (n, n - 3001):
        args = _args(rect, ntiles, depth, TX, TY, n, int(ntiles.sum()))
        args["n_vis"] = torch.tensor([n_vis], dtype=torch.int32, device="cuda")
        order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        H.hyrf_depth_order(n=n, pos=torch.as_tensor(pos, dtype=torch.float32).cuda(),
                           vis_ids=torch.arange(n, dtype=torch.int32, device="cuda"), n_vis=args["n_vis"],
                           cam=H.camera(cam), order=order, status=st)
        plain = _outputs(n, args["capacity"], TX * TY)
        H.hyrf_bin_sort(**args, **plain)  # without the depth order
        args["depth_order"] = order
        ref, got = _run_both(args, n, args["capacity"], TX * TY)
        K = int(ntiles[:n_vis].sum())
        assert H.read_status(st) == 0
        assert int(got["n_instances"].item()) == K
        _same(ref, got, K)
        _same(plain, got, K)


def test_noalloc_reports_overflow_like_workspace_version():
    """Capacity below the instance count: the same status word and clamped
    count as hyrf_bin_sort."""
    rect, ntiles, depth, (TX, TY) = _inputs(6, 5000, 257, 171)
    n, K = 5000, int(ntiles.sum())
    cap = K // 2
    ref, got = _run_both(_args(rect, ntiles, depth, TX, TY, n, cap), n, cap, TX * TY)
    assert H.read_status(ref["status"]) & H.HYRF_ERR_OVERFLOW
    assert H.read_status(got["status"]) == H.read_status(ref["status"])
    assert int(got["n_instances"].item()) == int(ref["n_instances"].item())
