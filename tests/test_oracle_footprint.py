"""Pins of the binning's opacity-aware footprint (oracle FP32 replay).

Eq. 1 skips a pixel where alpha = o exp(-q/2) < 1/255, q = d^T Sigma'^-1 d,
so a Gaussian can only show in tiles with a pixel centre at q <= 2 ln(255 o).
The footprint keeps those tiles (with a margin) and drops the rest of the
rectangle:

* its threshold t against numpy's logarithm (1.02 x 2 ln(255 o) + 0.05);
* brute force over every pixel centre of every tile of the rectangle: no
  tile with a pixel at q <= 2 ln(255 o) is dropped, and no kept tile lies
  entirely beyond q = t;
* the composited image (Eq. 1, FP64) from the footprint's tile lists equals
  the one from the whole rectangles exactly.
"""
import numpy as np

from paper_2509_17083_gb300 import synth


def _scene(rng, n, W, H):
    pos = np.stack([rng.uniform(-2.0, 2.0, n), rng.uniform(-1.4, 1.4, n), rng.uniform(1.5, 6.0, n)], 1)
    # anisotropic: one long axis per Gaussian
    s = np.exp(rng.uniform(-5.0, -2.0, (n, 3)))
    s[:, 0] *= np.exp(rng.uniform(0.0, 2.5, n))
    q = synth.random_quats(rng, n)
    o = 1.0 / (1.0 + np.exp(-rng.standard_normal(n) * 2.0))
    cam = synth.pinhole(W, H, 60.0)
    return pos.astype(np.float32), s.astype(np.float32), q, o.astype(np.float32), cam


def test_footprint_threshold_matches_log(orc):
    rng = np.random.default_rng(31)
    pos, s, q, o, cam = _scene(rng, 400, 160, 128)
    rect, nt, depth, flag, m2, foot = orc.project_f32_footprint(pos, s, q, cam, o)
    ok = (flag == 0) & (o >= 1.0 / 255.0) & (rect[:, 2] > rect[:, 0])
    t_ref = 1.02 * 2.0 * np.log(255.0 * o[ok].astype(np.float64)) + 0.05
    np.testing.assert_allclose(foot[ok, 3], t_ref, rtol=2e-6, atol=2e-6)
    assert np.all(foot[o < 1.0 / 255.0, 3] < 0)
    assert np.all(nt[o < 1.0 / 255.0] == 0)


def test_footprint_against_brute_force(orc):
    rng = np.random.default_rng(32)
    W, H = 240, 176
    pos, s, q, o, cam = _scene(rng, 300, W, H)
    rect, nt_rect, depth, flag = orc.project_f32(pos, s, q, cam)
    rect2, nt, depth2, flag2, m2, foot = orc.project_f32_footprint(pos, s, q, cam, o)
    assert np.array_equal(rect, rect2) and np.array_equal(depth.view(np.uint32), depth2.view(np.uint32))
    TX, TY = orc.tiles_of(W, H)
    keys, vals, ranges = orc.bin_sort(rect, depth, TX, TY, m2, foot)
    kept = set()
    for k, g in zip(keys, vals):
        kept.add((int(g), int(k >> np.uint64(32))))
    counted = np.bincount(vals, minlength=len(pos)) if len(vals) else np.zeros(len(pos), int)
    assert np.array_equal(counted, nt)
    assert nt.sum() < 0.8 * nt_rect.sum()  # the anisotropic scene drops a good share
    checked = dropped = 0
    for g in range(len(pos)):
        x0, y0, x1, y1 = rect[g]
        if x1 <= x0 or y1 <= y0:
            continue
        a, b, c, t = [float(x) for x in foot[g, :4]]
        Sg = np.array([[a, b], [b, c]])
        Q = np.linalg.inv(Sg)
        u, v = float(m2[g, 0]), float(m2[g, 1])
        t_true = 2.0 * np.log(255.0 * float(o[g])) if o[g] >= 1.0 / 255.0 else -1.0
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                xs = tx * 16 + 0.5 + np.arange(16)
                ys = ty * 16 + 0.5 + np.arange(16)
                dx, dy = np.meshgrid(xs - u, ys - v)
                qv = Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy
                shows = flag[g] == 1 or qv.min() <= t_true
                is_kept = (g, ty * TX + tx) in kept
                checked += 1
                if shows:
                    assert is_kept, (g, tx, ty, qv.min(), t_true)
                if is_kept and flag[g] == 0 and np.isfinite(t):
                    # kept tiles reach the ellipse q <= t at some point of the
                    # tile's pixel-centre box (continuous): check on a fine grid
                    fx = tx * 16 + 0.5 + np.linspace(0.0, 15.0, 61)
                    fy = ty * 16 + 0.5 + np.linspace(0.0, 15.0, 61)
                    ex, ey = np.meshgrid(fx - u, fy - v)
                    qf = Q[0, 0] * ex * ex + 2 * Q[0, 1] * ex * ey + Q[1, 1] * ey * ey
                    assert qf.min() <= t * (1.0 + 1e-3) + 0.05, (g, tx, ty, qf.min(), t)
                dropped += (not is_kept)
    assert checked > 1000 and dropped > 100, (checked, dropped)
    # the packed row spans (rectangles of <= 16 rows, <= 255 columns) list
    # exactly the kept tiles; other records carry zero span words
    words = foot[:, 4:].view(np.uint32)
    packed = 0
    for g in range(len(pos)):
        x0, y0, x1, y1 = rect[g]
        if x1 <= x0 or y1 <= y0 or y1 - y0 > 16 or x1 - x0 > 255:
            assert not words[g].any()
            continue
        packed += 1
        tiles = set()
        for j in range(y1 - y0):
            h = (int(words[g, j // 2]) >> (16 * (j % 2))) & 0xFFFF
            tiles |= {(y0 + j) * TX + x0 + (h & 0xFF) + k for k in range(h >> 8)}
        assert tiles == {tt for (gg, tt) in kept if gg == g}, g
        assert len(tiles) == nt[g]
    assert packed > 100


def test_footprint_lists_composite_like_rectangles(orc):
    rng = np.random.default_rng(33)
    W, H = 200, 144
    pos, s, q, o, cam = _scene(rng, 500, W, H)
    rect, _, depth, _ = orc.project_f32(pos, s, q, cam)
    _, nt, _, _, m2, foot = orc.project_f32_footprint(pos, s, q, cam, o)
    TX, TY = orc.tiles_of(W, H)
    mean2d, conic, _ = orc.project(pos.astype(np.float64), s.astype(np.float64), q.astype(np.float64), cam)
    col = rng.uniform(0.0, 1.0, (len(pos), 3))
    _, vr, rr = orc.bin_sort(rect, depth, TX, TY)
    _, vf, rf = orc.bin_sort(rect, depth, TX, TY, m2, foot)
    assert len(vf) < len(vr)
    Cr, Tr, _, _ = orc.rasterize(W, H, rr, vr, mean2d, conic, o.astype(np.float64), col)
    Cf, Tf, _, _ = orc.rasterize(W, H, rf, vf, mean2d, conic, o.astype(np.float64), col)
    assert np.array_equal(Cr, Cf) and np.array_equal(Tr, Tf)
