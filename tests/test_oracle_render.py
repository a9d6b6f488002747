"""Pins of the oracle's rendering stages: pre-cull (Eqs. 8-9), projection
(3DGS EWA conventions), binning, compositing (Eq. 1), background
(Eqs. 10-11, App. A.2) and loss (Eq. 12).

Every check compares the oracle with something independent of it: closed
forms, library routines (numpy eigvalsh, scipy rotations / correlate),
brute force, invariants, or central finite differences.
"""
import numpy as np
import pytest

from paper_2509_17083_gb300 import synth

sig = lambda x: 1.0 / (1.0 + np.exp(-x))


def _cam(W=64, H=48, f=60.0):
    return synth.pinhole(W, H, fx=f)


# ------------------------------------------------------------------ pre-cull

def test_precull_cases(orc):
    cam = _cam()  # W=64, H=48, fx=fy=60, cx=32, cy=24, tol 0.3, z_near 0.2
    # x_ndc = 2u/W - 1 with u = fx x/z + cx: |x_ndc| <= 1.3  <=>  |x/z| <= 1.3*32/60
    lim = 1.3 * 32 / 60
    pts = np.array([[0, 0, 1.0],          # on axis: kept
                    [0, 0, -1.0],         # behind: dropped
                    [0, 0, 0.1],          # closer than z_near: dropped
                    [lim * 0.99 * 2, 0, 2.0],   # inside the band: kept
                    [lim * 1.01 * 2, 0, 2.0],   # outside: dropped
                    [0, 1.3 * 24 / 60 * 0.98 * 5, 5.0],  # y inside: kept
                    [0, 1.3 * 24 / 60 * 1.02 * 5, 5.0]], np.float32)
    vis = orc.precull_f32(pts, cam)
    assert vis.tolist() == [True, False, False, True, False, True, False]


def test_precull_matches_fp64_away_from_the_boundary(orc):
    rng = np.random.default_rng(1)
    cam = synth.look_at([1, -0.5, -3], [0, 0, 2], 80, 60, 70.0)
    pts = rng.uniform(-4, 4, (5000, 3)).astype(np.float32)
    vis = orc.precull_f32(pts, cam)
    p = pts.astype(np.float64)
    tc = p @ cam.R.astype(np.float64).T + cam.t.astype(np.float64)
    z = tc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        xn = 2 * (cam.fx * tc[:, 0] / z + cam.cx) / cam.width - 1
        yn = 2 * (cam.fy * tc[:, 1] / z + cam.cy) / cam.height - 1
    ref = (z > 0.2) & (np.abs(xn) <= 1.3) & (np.abs(yn) <= 1.3)
    far = (np.abs(z - 0.2) > 1e-5) & (np.abs(np.abs(xn) - 1.3) > 1e-5) & (np.abs(np.abs(yn) - 1.3) > 1e-5)
    assert far.mean() > 0.99
    assert np.array_equal(vis[far], ref[far])


# ------------------------------------------------------------------ projection

def _sigma2d_reference(p, s, q_wxyz, cam):
    """Sigma' = J Sigma J^T + 0.3 I with J the finite-difference Jacobian of
    (u, v) = (fx x/z + cx, fy y/z + cy) and Sigma from scipy's rotation."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    Rq = Rot.from_quat([q_wxyz[1], q_wxyz[2], q_wxyz[3], q_wxyz[0]]).as_matrix()
    Sig = Rq @ np.diag(np.asarray(s) ** 2) @ Rq.T
    Rc = cam.R.astype(np.float64)
    tc = Rc @ p + cam.t

    def uv(t):
        return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])
    J = np.zeros((2, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = 1e-6
        J[:, j] = (uv(tc + e) - uv(tc - e)) / 2e-6
    Sig_c = Rc @ Sig @ Rc.T
    return J @ Sig_c @ J.T + 0.3 * np.eye(2), uv(tc), tc[2]


def test_project_isotropic_on_axis_closed_form(orc):
    cam = _cam()
    s, z = 0.05, 2.5
    m, con, d = orc.project(np.array([[0, 0, z]]), np.array([[s, s, s]]),
                            np.array([[1.0, 0, 0, 0]]), cam)
    v = (cam.fx * s / z) ** 2 + 0.3
    np.testing.assert_allclose(m[0], [cam.cx, cam.cy], atol=1e-12)
    np.testing.assert_allclose(con[0], [1 / v, 0, 1 / v], rtol=1e-13, atol=1e-15)
    assert d[0] == z


def test_project_general_matches_reference(orc):
    rng = np.random.default_rng(2)
    cam = synth.look_at([0.5, -1, -2], [0, 0, 3], 96, 64, 60.0)
    n = 40
    pos = rng.uniform([-1, -1, 2], [1, 1, 4], (n, 3))
    s = np.exp(rng.uniform(-4, -1, (n, 3)))
    q = synth.random_quats(rng, n).astype(np.float64)
    m, con, d = orc.project(pos, s, q, cam)
    for i in range(n):
        S2, uv, z = _sigma2d_reference(pos[i], s[i], q[i], cam)
        tx = (cam.R.astype(np.float64) @ pos[i] + cam.t)
        if abs(tx[0] / tx[2]) > 1.3 * 48 / cam.fx or abs(tx[1] / tx[2]) > 1.3 * 32 / cam.fy:
            continue  # outside the clamp: J differs from the plain derivative
        inv = np.linalg.inv(S2)
        np.testing.assert_allclose(con[i], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(m[i], uv, rtol=1e-12)
        np.testing.assert_allclose(d[i], z, rtol=1e-12)


def test_project_fp32_rect_matches_fp64_definition(orc):
    rng = np.random.default_rng(3)
    cam = synth.pinhole(200, 120, 60.0)
    n = 3000
    pos = np.stack([rng.uniform(-2, 2, n), rng.uniform(-1.2, 1.2, n), rng.uniform(1.5, 6, n)], 1)
    s = np.exp(rng.uniform(-5, -1.5, (n, 3)))
    q = synth.random_quats(rng, n)
    p32, s32, q32 = pos.astype(np.float32), s.astype(np.float32), q.astype(np.float32)
    rect, ntiles, depth, flag = orc.project_f32(p32, s32, q32, cam, 16)
    m, con, d = orc.project(p32.astype(np.float64), s32.astype(np.float64), q32.astype(np.float64), cam)
    TX, TY = (200 + 15) // 16, (120 + 15) // 16
    checked = 0
    for i in range(n):
        inv = np.array([[con[i, 0], con[i, 1]], [con[i, 1], con[i, 2]]])
        lam = np.linalg.eigvalsh(np.linalg.inv(inv)).max()
        r = 3 * np.sqrt(lam)
        if abs(r - np.round(r)) < 1e-4:
            continue
        r = np.ceil(r)
        lo = (m[i] - r) / 16
        hi = (m[i] + r) / 16
        if np.any(np.abs(lo - np.round(lo)) < 1e-4) or np.any(np.abs(hi - np.round(hi)) < 1e-4):
            continue
        x0, y0 = np.clip(np.floor(lo), 0, [TX, TY])
        x1, y1 = np.clip(np.floor(hi) + 1, 0, [TX, TY])
        assert rect[i].tolist() == [x0, y0, x1, y1], i
        nt = (x1 - x0) * (y1 - y0) if (x1 > x0 and y1 > y0) else 0
        assert ntiles[i] == nt
        checked += 1
    assert checked > 0.99 * n
    np.testing.assert_array_equal(depth, d.astype(np.float32))
    # near-singular flag: |det| < 1e-2 a c of Sigma'
    assert flag.sum() < n


def test_project_backward_matches_finite_differences(orc):
    rng = np.random.default_rng(4)
    cam = synth.look_at([0.3, -0.4, -1.5], [0, 0, 3], 64, 48, 60.0)
    n = 12
    pos = rng.uniform([-0.8, -0.6, 2], [0.8, 0.6, 4], (n, 3))
    pos[0] = [3.0, 0.1, 2.0]  # outside the tangent clamp on x
    s = np.exp(rng.uniform(-3, -1, (n, 3)))
    q = synth.random_quats(rng, n).astype(np.float64) * rng.uniform(0.5, 2.0, (n, 1))
    wm, wc = rng.standard_normal((n, 2)), rng.standard_normal((n, 3))

    def L():
        m, c, _ = orc.project(pos, s, q, cam)
        return (wm * m).sum() + (wc * c).sum()
    dp, ds, dq = orc.project_backward(pos, s, q, cam, wm, wc)
    for arr, g in [(pos, dp), (s, ds), (q, dq)]:
        for i in range(n):
            for k in range(arr.shape[1]):
                v = arr[i, k]
                h = 1e-6 * max(1.0, abs(v))
                arr[i, k] = v + h
                lp = L()
                arr[i, k] = v - h
                lm = L()
                arr[i, k] = v
                np.testing.assert_allclose(g[i, k], (lp - lm) / (2 * h), rtol=2e-5, atol=1e-7)


# ------------------------------------------------------------------ binning and compositing

def _scene(rng, n, W, H, s_range=(-4, -1.5)):
    cam = synth.pinhole(W, H, 60.0)
    pos = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(-1, 1, n), rng.uniform(2, 5, n)], 1)
    s = np.exp(rng.uniform(*s_range, (n, 3)))
    q = synth.random_quats(rng, n).astype(np.float64)
    m, con, d = orc_project(pos, s, q, cam)
    return cam, pos, s, q, m, con


def orc_project(pos, s, q, cam):
    import oracle
    return oracle.project(pos, s, q, cam)


def test_binning_and_tiled_equals_untiled(orc):
    rng = np.random.default_rng(5)
    W, H = 70, 50
    n = 300
    cam, pos, s, q, m, con = _scene(rng, n, W, H)
    rect, ntiles, d32, _ = orc.project_f32(pos, s, q, cam)
    TX, TY = orc.tiles_of(W, H)
    keys, vals, ranges = orc.bin_sort(rect, d32, TX, TY)
    assert len(keys) == ntiles.sum()
    assert np.all(keys[1:] >= keys[:-1])
    # every Gaussian appears in exactly its rectangle's tiles
    for g in range(n):
        tiles = sorted((keys[vals == g] >> np.uint64(32)).astype(int).tolist())
        r = rect[g]
        exp = sorted(ty * TX + tx for ty in range(r[1], r[3]) for tx in range(r[0], r[2]))
        assert tiles == exp
    for t in range(TX * TY):
        a, b = ranges[t]
        assert np.all((keys[a:b] >> np.uint64(32)) == t)
    op = sig(rng.standard_normal(n))
    col = rng.uniform(0, 1, (n, 3))
    C1, T1, _, _ = orc.rasterize(W, H, ranges, vals, m, con, op, col)
    C2, T2 = orc.rasterize_untiled(W, H, rect, d32, m, con, op, col)
    assert np.array_equal(C1, C2) and np.array_equal(T1, T2)
    assert (T1 < 1).mean() > 0.5


def test_single_gaussian_closed_form(orc):
    W, H = 40, 32
    m = np.array([[17.3, 14.1]])
    con = np.array([[0.05, 0.01, 0.08]])
    op = np.array([0.8])
    col = np.array([[0.2, 0.5, 0.9]])
    ranges = np.zeros((3 * 2, 2), np.int32)
    TX, TY = orc.tiles_of(W, H)
    ranges = np.zeros((TX * TY, 2), np.int32)
    vals = np.zeros(TX * TY, np.int32)
    for t in range(TX * TY):
        ranges[t] = [t, t + 1]
    C, T, nc, _ = orc.rasterize(W, H, ranges, vals, m, con, op, col)
    ys, xs = np.mgrid[0:H, 0:W]
    dx, dy = m[0, 0] - (xs + 0.5), m[0, 1] - (ys + 0.5)
    a = np.minimum(0.99, op[0] * np.exp(-0.5 * (con[0, 0] * dx ** 2 + con[0, 2] * dy ** 2) - con[0, 1] * dx * dy))
    a = np.where(a < 1 / 255, 0.0, a)
    np.testing.assert_allclose(T, 1 - a, atol=1e-15)
    np.testing.assert_allclose(C, a[..., None] * col[0], atol=1e-15)


def test_two_gaussians_composite_front_to_back(orc):
    """Eq. 1 for two overlapping Gaussians binned and depth-sorted together:
    C = c_n a_n + c_f a_f (1 - a_n) and T = (1 - a_n)(1 - a_f) at every pixel,
    with n the nearer one whatever the input order; swapping the depths swaps
    the roles."""
    W, H = 40, 32
    TX, TY = orc.tiles_of(W, H)
    m = np.array([[15.2, 13.7], [21.9, 17.4]])
    con = np.array([[0.02, 0.004, 0.03], [0.03, -0.006, 0.025]])
    op = np.array([0.7, 0.8])
    col = np.array([[0.9, 0.2, 0.1], [0.1, 0.3, 0.95]])
    rect = np.array([[0, 0, TX, TY]] * 2, np.int32)
    ys, xs = np.mgrid[0:H, 0:W]

    def alpha(g):
        dx, dy = m[g, 0] - (xs + 0.5), m[g, 1] - (ys + 0.5)
        a = np.minimum(0.99, op[g] * np.exp(-0.5 * (con[g, 0] * dx ** 2 + con[g, 2] * dy ** 2)
                                            - con[g, 1] * dx * dy))
        return np.where(a < 1 / 255, 0.0, a)
    for depths, near, far in (([5.0, 2.0], 1, 0), ([2.0, 5.0], 0, 1)):
        _, vals, ranges = orc.bin_sort(rect, np.array(depths, np.float32), TX, TY)
        C, T, _, _ = orc.rasterize(W, H, ranges, vals, m, con, op, col)
        an, af = alpha(near), alpha(far)
        np.testing.assert_allclose(T, (1 - an) * (1 - af), atol=1e-15)
        np.testing.assert_allclose(C, an[..., None] * col[near] + (af * (1 - an))[..., None] * col[far],
                                   atol=1e-14)
        assert (an * af > 0.1).sum() > 20  # the two overlap


def test_weights_sum_to_one_minus_T(orc):
    rng = np.random.default_rng(6)
    W, H = 64, 48
    n = 400
    cam, pos, s, q, m, con = _scene(rng, n, W, H, (-3, -1))
    rect, ntiles, d32, _ = orc.project_f32(pos, s, q, cam)
    TX, TY = orc.tiles_of(W, H)
    keys, vals, ranges = orc.bin_sort(rect, d32, TX, TY)
    op = sig(rng.standard_normal(n) + 2)
    C, T, nc, _ = orc.rasterize(W, H, ranges, vals, m, con, op, np.ones((n, 3)))
    np.testing.assert_allclose(C, np.repeat((1 - T)[..., None], 3, -1), atol=1e-12)
    assert T.min() >= 1e-4 * (1 - 0.99) and T.max() <= 1.0
    assert (nc > 0).mean() > 0.5


def test_rasterize_backward_matches_finite_differences(orc):
    rng = np.random.default_rng(7)
    W, H = 48, 32
    n = 60
    cam, pos, s, q, m, con = _scene(rng, n, W, H, (-3, -1.5))
    rect, ntiles, d32, _ = orc.project_f32(pos, s, q, cam)
    TX, TY = orc.tiles_of(W, H)
    keys, vals, ranges = orc.bin_sort(rect, d32, TX, TY)
    op = sig(rng.standard_normal(n))
    op[:3] = 0.9999  # alpha clamped at 0.99 near the centre of these
    col = rng.uniform(0, 1, (n, 3))
    C0, T0, nc0, mg = orc.rasterize(W, H, ranges, vals, m, con, op, col)
    wC = rng.standard_normal((H, W, 3)) * (mg > 1e-4)[..., None]
    wT = rng.standard_normal((H, W)) * (mg > 1e-4)

    def L():
        C, T, _, _ = orc.rasterize(W, H, ranges, vals, m, con, op, col)
        return (wC * C).sum() + (wT * T).sum()
    dm, dc, do, dcol = orc.rasterize_backward(W, H, ranges, vals, m, con, op, col, wC, wT)
    for arr, g in [(m, dm), (con, dc), (op.reshape(-1, 1), do.reshape(-1, 1)), (col, dcol)]:
        for i in rng.choice(n, 15, replace=False):
            for k in range(arr.shape[1]):
                v = arr[i, k]
                h = 1e-7 * max(1.0, abs(v))
                arr[i, k] = v + h
                lp = L()
                arr[i, k] = v - h
                lm = L()
                arr[i, k] = v
                np.testing.assert_allclose(g[i, k], (lp - lm) / (2 * h), rtol=1e-4, atol=1e-7)


# ------------------------------------------------------------------ background

def test_ray_sphere_hit(orc):
    cam = synth.look_at([2, -1, -5], [0, 0, 3], 32, 24, 60.0)
    lo, hi = np.array([-3.0, -2, 0]), np.array([3.0, 2, 8])
    for (i, j) in [(0, 0), (31, 23), (15, 11), (3, 20)]:
        ps, t, o, d = orc.ray_sphere(cam, lo, hi, 100.0, i, j)
        assert t > 0
        np.testing.assert_allclose(np.linalg.norm(ps), 100.0, rtol=1e-13)
        np.testing.assert_allclose(ps, o + t * d, rtol=1e-13)
        # o is the camera centre in normalised coordinates
        np.testing.assert_allclose(o, 2 * (cam.center() - lo) / (hi - lo) - 1, atol=1e-6)


def _bg_fields(rng, const_bias=None):
    fl = synth.make_fields(rng, [-2, -2, 1], [2, 2, 6], 4, 8, 16, 2, 0.5, pe_freq=2, pe_pad=16)
    if const_bias is not None:
        fl.col_mlp.W = [np.zeros_like(w) for w in fl.col_mlp.W]
        fl.col_mlp.b[-1] = np.asarray(const_bias, np.float32)
    return fl


@pytest.mark.parametrize("mode", [0, 1])
def test_background_constant_field(orc, mode):
    rng = np.random.default_rng(8)
    b = [0.4, -1.2, 2.0]
    fl = _bg_fields(rng, b)
    cam = synth.look_at([0.2, 0.1, -2], [0, 0, 3], 24, 16, 70.0)
    bg = synth.Background(mode, 8, 16)
    Cfg = rng.uniform(0, 1, (16, 24, 3))
    T = rng.uniform(0, 1, (16, 24))
    C, cs = orc.background(cam, fl, bg, Cfg, T)
    bb = np.array(b, np.float32).astype(np.float64)
    np.testing.assert_allclose(cs, np.broadcast_to(sig(bb), cs.shape), rtol=1e-12)
    np.testing.assert_allclose(C, Cfg + T[..., None] * sig(bb), rtol=1e-12)


@pytest.mark.parametrize("mode", [0, 1])
def test_background_depends_on_the_world_ray_only(orc, mode):
    """Eq. 10 queries the field along the pixel's world-space ray. A camera
    rolled by 180 degrees about its optical axis (camera x and y negated;
    principal point at the image centre) sees at pixel (W-1-i, H-1-j) the
    ray of pixel (i, j): same centre, same world direction, so the same
    background colour. A positional encoding of the camera-space direction,
    or a ray origin taken from t alone, would break it."""
    rng = np.random.default_rng(12)
    fl = _bg_fields(rng)
    cam = synth.look_at([0.2, 0.1, -2], [0, 0, 3], 24, 16, 70.0)
    flip = np.diag([-1.0, -1.0, 1.0]).astype(np.float32)
    rolled = synth.pinhole(24, 16, fx=cam.fx, R=flip @ cam.R, t=flip @ cam.t)
    bg = synth.Background(mode, 8, 16)
    Cfg, T = np.zeros((16, 24, 3)), np.ones((16, 24))
    _, ca = orc.background(cam, fl, bg, Cfg, T)
    _, cb = orc.background(rolled, fl, bg, Cfg, T)
    np.testing.assert_allclose(cb, ca[::-1, ::-1], rtol=1e-12, atol=1e-14)
    assert np.abs(ca - ca[::-1, ::-1]).max() > 1e-3  # the view itself is not symmetric


def test_background_map_converges_to_exact_mode(orc):
    """Map-mode geometry (texel centres, the longitude and latitude axes,
    bilinear weights) against the exact mode: seen from the centre of a cubic
    box, a pixel's sphere hit lies along its own ray, so the map colour is the
    bilinear interpolation, over the texel directions, of the colour the exact
    mode gives that ray. For a smooth colour field the error falls as O(h^2),
    about 4x per halving of the texel size. A half-texel offset gives O(h)
    (ratios near 0.5), and a swapped or mirrored axis does not converge."""
    rng = np.random.default_rng(21)
    fl = synth.make_fields(rng, [-2, -2, -2], [2, 2, 2], 4, 8, 16, 2, 0.5, pe_freq=2, pe_pad=16)
    fl.rad.table = np.zeros_like(fl.rad.table)  # the colour depends on the direction only
    m = fl.col_mlp
    # positive pre-activations in every hidden unit: a smooth colour field
    m.W = [rng.uniform(-0.05, 0.05, w.shape).astype(np.float32) for w in m.W[:-1]] + \
        [rng.uniform(-1, 1, m.W[-1].shape).astype(np.float32)]
    m.b = [np.full_like(b, 4.0) for b in m.b[:-1]] + [np.zeros_like(m.b[-1])]
    cam = synth.look_at([0, 0, 0], [0.1, 0.05, 1], 24, 16, 60.0)  # the box centre
    Cfg, T = np.zeros((16, 24, 3)), np.ones((16, 24))
    _, ce = orc.background(cam, fl, synth.Background(0, 0, 0, 100.0), Cfg, T)
    assert np.ptp(ce) > 0.5  # the colour varies over the view
    errs = []
    for mh in (16, 32, 64, 128):
        _, cm = orc.background(cam, fl, synth.Background(1, mh, 2 * mh, 100.0), Cfg, T)
        errs.append(np.abs(cm - ce).max())
    ratios = np.array(errs[1:]) / np.array(errs[:-1])
    assert np.all((ratios > 0.15) & (ratios < 0.35)), (errs, ratios)
    assert errs[-1] < 1e-5


@pytest.mark.parametrize("mode", [0, 1])
def test_background_backward_matches_finite_differences(orc, mode):
    rng = np.random.default_rng(9)
    fl = _bg_fields(rng)
    fl.rad.table = fl.rad.table.astype(np.float64)
    fl.col_mlp.W = [w.astype(np.float64) for w in fl.col_mlp.W]
    cam = synth.look_at([0.2, 0.1, -2], [0, 0, 3], 20, 14, 70.0)
    bg = synth.Background(mode, 6, 12)
    Cfg = rng.uniform(0, 1, (14, 20, 3))
    T = rng.uniform(0, 1, (14, 20))
    wC = rng.standard_normal((14, 20, 3))

    def L():
        C, _ = orc.background(cam, fl, bg, Cfg, T)
        return (wC * C).sum()
    g = orc.background_backward(cam, fl, bg, T, wC)
    np.testing.assert_array_equal(g["C_fg"], wC)

    def fd(arr, e):
        v = arr[e]
        h = 1e-6 * max(1, abs(v))
        arr[e] = v + h
        lp = L()
        arr[e] = v - h
        lm = L()
        arr[e] = v
        return (lp - lm) / (2 * h)
    for e in [(0, 0), (5, 7), (13, 19), (7, 3)]:
        np.testing.assert_allclose(g["T_final"][e], fd(T, e), rtol=1e-6, atol=1e-9)
    nz = np.argwhere(np.abs(g["rad_table"]) > 1e-8)
    for e in nz[rng.choice(len(nz), 10, replace=False)]:
        e = tuple(e)
        np.testing.assert_allclose(g["rad_table"][e], fd(fl.rad.table, e), rtol=1e-5, atol=1e-9)
    for l in range(3):
        W = fl.col_mlp.W[l]
        for _ in range(3):
            e = (rng.integers(W.shape[0]), rng.integers(W.shape[1]))
            np.testing.assert_allclose(g["col_W"][l][e], fd(W, e), rtol=1e-5, atol=1e-9)


# ------------------------------------------------------------------ loss

def test_ssim_identity_and_library_reference(orc):
    nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(10)
    x = rng.uniform(0, 1, (23, 31, 3))
    y = np.clip(x + 0.1 * rng.standard_normal(x.shape), 0, 1)
    np.testing.assert_allclose(orc.ssim(x, x), 1.0, atol=1e-13)
    g1 = np.exp(-((np.arange(11) - 5) ** 2) / (2 * 1.5 ** 2))
    g1 /= g1.sum()
    k = np.outer(g1, g1)
    tot = 0
    for ch in range(3):
        a, b = x[..., ch], y[..., ch]
        f = lambda im: nd.correlate(im, k, mode="constant", cval=0.0)
        mx, my = f(a), f(b)
        vx, vy, cxy = f(a * a) - mx ** 2, f(b * b) - my ** 2, f(a * b) - mx * my
        C1, C2 = 0.01 ** 2, 0.03 ** 2
        tot += (((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx ** 2 + my ** 2 + C1) * (vx + vy + C2))).mean()
    np.testing.assert_allclose(orc.ssim(x, y), tot / 3, rtol=1e-12)


def test_l1_closed_form(orc):
    rng = np.random.default_rng(11)
    x, y = rng.uniform(0, 1, (7, 9, 3)), rng.uniform(0, 1, (7, 9, 3))
    L, dC = orc.loss(x, y, 0.0)
    np.testing.assert_allclose(L, np.abs(x - y).mean(), rtol=1e-14)
    np.testing.assert_allclose(dC, np.sign(x - y) / x.size, rtol=1e-14)


def test_loss_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(12)
    x, y = rng.uniform(0, 1, (13, 17, 3)), rng.uniform(0, 1, (13, 17, 3))
    L0, dC = orc.loss(x, y, 0.2)
    for _ in range(25):
        e = (rng.integers(13), rng.integers(17), rng.integers(3))
        v = x[e]
        h = 1e-6
        x[e] = v + h
        lp = orc.loss(x, y, 0.2)[0]
        x[e] = v - h
        lm = orc.loss(x, y, 0.2)[0]
        x[e] = v
        np.testing.assert_allclose(dC[e], (lp - lm) / (2 * h), rtol=1e-5, atol=1e-10)
