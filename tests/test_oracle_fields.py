"""Pins of the oracle's neural-field stage (Sec. 3.2, Eqs. 2-7; App. A.1).

Each test checks the oracle against something other than itself: closed
forms, special cases that reduce to a library routine, published constants,
or central finite differences of the oracle's own forward pass.
"""
import numpy as np
import pytest

from paper_2509_17083_gb300 import synth

BOX_LO = np.array([-1.0, -2.0, 1.0])
BOX_HI = np.array([3.0, 2.0, 5.0])


def _p_from_x(x):
    """World point whose App. A.1 normalisation is x."""
    return BOX_LO + (np.asarray(x) + 1.0) * (BOX_HI - BOX_LO) / 2.0


def test_contraction_closed_form(orc):
    # inside the unit ball: y = 0.25 x + 0.5
    y, _ = orc.contract(BOX_LO, BOX_HI, _p_from_x([0.2, -0.4, 0.6]))
    np.testing.assert_allclose(y, [0.55, 0.4, 0.65], rtol=0, atol=1e-15)
    # outside: |x| = 2 along +x -> 0.25 * (2 - 1/2) * 1 + 0.5 = 0.875
    y, _ = orc.contract(BOX_LO, BOX_HI, _p_from_x([2.0, 0.0, 0.0]))
    np.testing.assert_allclose(y, [0.875, 0.5, 0.5], atol=1e-15)
    # |x| = 4 along -z -> 0.5 - 0.25 * (2 - 1/4) = 0.0625
    y, _ = orc.contract(BOX_LO, BOX_HI, _p_from_x([0.0, 0.0, -4.0]))
    np.testing.assert_allclose(y, [0.5, 0.5, 0.0625], atol=1e-15)


def test_contraction_range_and_continuity(orc):
    rng = np.random.default_rng(3)
    for _ in range(200):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        r = 10 ** rng.uniform(-2, 6)
        y, _ = orc.contract(BOX_LO, BOX_HI, _p_from_x(d * r))
        assert np.all(y > 0.0) and np.all(y < 1.0), (r, y)
    # C^1 at |x| = 1: value and Jacobian agree from both sides
    d = np.array([0.48, -0.6, 0.64])
    d /= np.linalg.norm(d)
    ya, Ja = orc.contract(BOX_LO, BOX_HI, _p_from_x(d * (1 - 1e-9)))
    yb, Jb = orc.contract(BOX_LO, BOX_HI, _p_from_x(d * (1 + 1e-9)))
    np.testing.assert_allclose(ya, yb, atol=1e-8)
    np.testing.assert_allclose(Ja, Jb, atol=1e-7)


def test_contraction_jacobian_fd(orc):
    rng = np.random.default_rng(4)
    for r in [0.5, 1.7, 30.0]:
        d = rng.standard_normal(3)
        p = _p_from_x(d / np.linalg.norm(d) * r)
        _, J = orc.contract(BOX_LO, BOX_HI, p)
        Jfd = np.zeros((3, 3))
        for j in range(3):
            h = 1e-6 * max(1, abs(p[j]))
            e = np.zeros(3)
            e[j] = h
            Jfd[:, j] = (orc.contract(BOX_LO, BOX_HI, p + e)[0] - orc.contract(BOX_LO, BOX_HI, p - e)[0]) / (2 * h)
        np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-9)


def test_level_resolutions(orc):
    g = synth.HashGrid(16, 19, np.zeros((16, 1 << 19, 2), np.float32))
    res = [orc.level_res(g, l) for l in range(16)]
    # floor(16 * 1.5^l), hand-evaluated
    assert res == [16, 24, 36, 54, 81, 121, 182, 273, 410, 615, 922, 1383, 2075, 3113, 4670, 7006]


def test_dense_hashed_switch(orc):
    # level 0 of base 16 has 17^3 = 4913 vertices: dense iff T >= 4913
    for log2T, dense in [(12, False), (13, True)]:
        g = synth.HashGrid(1, log2T, np.zeros((1, 1 << log2T, 2), np.float32))
        idx = orc.level_index(g, 0, 3, 5, 7)
        if dense:
            assert idx == 3 + 5 * 17 + 7 * 17 * 17
        else:
            # Instant-NGP spatial hash, primes (1, 2654435761, 805459861), mod 2^32
            h = (3 * 1) ^ ((5 * 2654435761) % 2**32) ^ ((7 * 805459861) % 2**32)
            assert idx == h % (1 << log2T)


def test_hash_trilinear_reproduces_linear_function(orc):
    # Dense level: a table holding a*ix + b*iy + c*iz + d at vertex (ix,iy,iz)
    # is reproduced exactly by trilinear interpolation: a*u + b*v + c*w + d.
    N = 16
    log2T = 13
    g = synth.HashGrid(1, log2T, np.zeros((1, 1 << log2T, 2), np.float32), base_res=N)
    tab = np.zeros((1, 1 << log2T, 2))
    coef = np.array([[0.3, -0.7, 1.1, 0.25], [-2.0, 0.5, 0.125, -1.0]])
    for iz in range(N + 1):
        for iy in range(N + 1):
            for ix in range(N + 1):
                e = ix + iy * (N + 1) + iz * (N + 1) ** 2
                tab[0, e] = coef[:, 0] * ix + coef[:, 1] * iy + coef[:, 2] * iz + coef[:, 3]
    g.table = tab
    rng = np.random.default_rng(5)
    for _ in range(50):
        y = rng.uniform(0.001, 0.999, 3)
        u = y * N
        f = orc.hash_encode(g, y)
        np.testing.assert_allclose(f, coef[:, :3] @ u + coef[:, 3], rtol=1e-12, atol=1e-12)


def test_hash_partition_of_unity(orc):
    # constant table -> every level returns that constant (weights sum to 1)
    g = synth.HashGrid(8, 10, np.zeros((8, 1024, 2)))
    g.table = np.broadcast_to(np.array([0.375, -1.5]), (8, 1024, 2)).copy()
    rng = np.random.default_rng(6)
    for _ in range(20):
        f = orc.hash_encode(g, rng.uniform(0, 1, 3))
        np.testing.assert_allclose(f.reshape(8, 2), np.tile([0.375, -1.5], (8, 1)), atol=1e-14)


def test_mlp_matches_numpy(orc):
    rng = np.random.default_rng(7)
    m = synth.xavier_mlp(rng, 48, 32, 1, 3)
    m.b = [rng.standard_normal(len(b)) for b in m.b]
    for n_hidden, width, n_in in [(1, 32, 48), (2, 64, 64)]:
        m = synth.xavier_mlp(rng, n_in, width, n_hidden, 8)
        m.b = [rng.standard_normal(len(b)).astype(np.float32) for b in m.b]
        x = rng.standard_normal(n_in)
        h = x
        for l in range(n_hidden):
            h = np.maximum(m.W[l].astype(np.float64) @ h + m.b[l], 0.0)
        ref = m.W[-1].astype(np.float64) @ h + m.b[-1]
        np.testing.assert_allclose(orc.mlp_forward(m, x), ref, rtol=1e-12, atol=1e-12)


def test_positional_encoding_closed_form(orc):
    pe = orc.pos_enc([1.0, 0.0, 0.5], 4)
    assert len(pe) == 27
    np.testing.assert_allclose(pe[:3], [1.0, 0.0, 0.5])
    # k = 0: sin(pi*[1,0,.5]) = [0,0,1], cos = [-1,1,0]
    np.testing.assert_allclose(pe[3:9], [0, 0, 1, -1, 1, 0], atol=1e-15)
    # k = 1: sin(2 pi [1,0,.5]) = 0, cos = [1,1,-1]
    np.testing.assert_allclose(pe[9:15], [0, 0, 0, 1, 1, -1], atol=1e-15)
    # k = 3: 8 pi * 0.5 = 4 pi
    np.testing.assert_allclose(pe[21:27], [0, 0, 0, 1, 1, 1], atol=1e-14)


def _small_fields(rng, table_init=0.5, n_levels=4, log2_T=8, width=16, n_hidden=2):
    return synth.make_fields(rng, BOX_LO, BOX_HI, n_levels, log2_T, width, n_hidden, table_init,
                             pe_freq=2, pe_pad=16)


def test_query_reduces_to_bias_when_weights_vanish(orc):
    rng = np.random.default_rng(8)
    fl = _small_fields(rng)
    for m in (fl.geo_mlp, fl.col_mlp):
        m.W = [np.zeros_like(w) for w in m.W]
    fl.geo_mlp.b[-1] = np.array([0.3, -0.2, 0.1, 0.4, 2.0, -1.0, 0.5, 1.0], np.float32)
    fl.col_mlp.b[-1] = np.array([0.7, -0.1, 0.2], np.float32)
    n = 5
    pos = rng.uniform(-1, 3, (n, 3))
    ae, se, ce = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal((n, 3))
    cam = synth.pinhole(64, 64, 60.0)
    a, s, q, c = orc.query_fields(pos, ae, se, ce, cam, fl)
    sig = lambda x: 1 / (1 + np.exp(-x))
    b = fl.geo_mlp.b[-1].astype(np.float64)
    np.testing.assert_allclose(a, sig(b[0] + ae), rtol=1e-14)
    np.testing.assert_allclose(s, sig(b[1:4][None] + se[:, None]), rtol=1e-14)
    np.testing.assert_allclose(q, np.tile(b[4:] / np.linalg.norm(b[4:]), (n, 1)), rtol=1e-14)
    np.testing.assert_allclose(c, sig(fl.col_mlp.b[-1].astype(np.float64)[None] + ce), rtol=1e-14)


def test_query_depends_on_the_camera_centre_only(orc):
    """The colour decoder's view direction (Eq. 6) runs from the camera centre
    to the Gaussian in world space, and the geometry decoder sees no camera:
    a camera rolled by 180 degrees about its optical axis (same centre) gives
    the same outputs for every Gaussian, while moving the centre changes the
    colours. The camera-space direction would fail the first check."""
    rng = np.random.default_rng(14)
    fl = _small_fields(rng)
    n = 16
    pos = rng.uniform(-1, 3, (n, 3))
    ae, se, ce = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal((n, 3))
    cam = synth.look_at([0.5, -0.3, -4], [1, 1, 1], 64, 48, 60.0)
    flip = np.diag([-1.0, -1.0, 1.0]).astype(np.float32)
    rolled = synth.pinhole(64, 48, fx=cam.fx, R=flip @ cam.R, t=flip @ cam.t)
    out_a = orc.query_fields(pos, ae, se, ce, cam, fl)
    out_b = orc.query_fields(pos, ae, se, ce, rolled, fl)
    for x, y in zip(out_a, out_b):
        np.testing.assert_allclose(y, x, rtol=1e-12, atol=1e-15)
    moved = synth.look_at([2.5, -0.3, -4], [1, 1, 1], 64, 48, 60.0)
    out_c = orc.query_fields(pos, ae, se, ce, moved, fl)
    for x, y in zip(out_a[:3], out_c[:3]):
        np.testing.assert_allclose(y, x, rtol=1e-12, atol=1e-15)  # geometry: no camera
    assert np.abs(out_c[3] - out_a[3]).max() > 1e-4  # colour: the direction changed


def test_query_backward_matches_finite_differences(orc):
    rng = np.random.default_rng(9)
    fl = _small_fields(rng)
    for m in (fl.geo_mlp, fl.col_mlp):
        m.b = [rng.standard_normal(len(b)).astype(np.float32) * 0.3 for b in m.b]
    n = 6
    pos = rng.uniform(-1, 3, (n, 3))
    pos[0] = [20.0, -30.0, 50.0]  # a point in the contracted (outer) region
    ae, se, ce = rng.standard_normal(n), rng.standard_normal(n), rng.standard_normal((n, 3))
    cam = synth.pinhole(64, 64, 60.0, R=synth.look_at([5, 1, -3], [1, 0, 3], 64, 64, 60).R,
                        t=synth.look_at([5, 1, -3], [1, 0, 3], 64, 64, 60).t)
    wa, ws, wq, wc = rng.standard_normal(n), rng.standard_normal((n, 3)), \
        rng.standard_normal((n, 4)), rng.standard_normal((n, 3))

    def L(pos=pos, ae=ae, se=se, ce=ce, fields=fl):
        a, s, q, c = orc.query_fields(pos, ae, se, ce, cam, fields)
        return (wa * a).sum() + (ws * s).sum() + (wq * q).sum() + (wc * c).sum()

    g = orc.query_fields_backward(pos, ae, se, ce, cam, fl, wa, ws, wq, wc)

    def fd(getter, setter, h=1e-6):
        v = getter()
        setter(v + h)
        lp = L()
        setter(v - h)
        lm = L()
        setter(v)
        return (lp - lm) / (2 * h)

    for i in range(n):
        for k in range(3):
            def st(v, i=i, k=k):
                pos[i, k] = v
            np.testing.assert_allclose(g["pos"][i, k], fd(lambda: pos[i, k], st), rtol=2e-5, atol=1e-8)
        for arr, key in [(ae, "alpha_e"), (se, "scale_e")]:
            def st(v, arr=arr, i=i):
                arr[i] = v
            np.testing.assert_allclose(g[key][i], fd(lambda: arr[i], st), rtol=1e-6, atol=1e-9)
        for k in range(3):
            def st(v, i=i, k=k):
                ce[i, k] = v
            np.testing.assert_allclose(g["color_e"][i, k], fd(lambda: ce[i, k], st), rtol=1e-6, atol=1e-9)
    # table entries that received gradient, and a few MLP weights
    for key, grid in [("geo_table", fl.geo), ("rad_table", fl.rad)]:
        grid.table = grid.table.astype(np.float64)
        gt = g[key]
        nz = np.argwhere(np.abs(gt) > 1e-6)
        for e in nz[rng.choice(len(nz), 8, replace=False)]:
            e = tuple(e)
            tab = grid.table

            def st(v, tab=tab, e=e):
                tab[e] = v
            np.testing.assert_allclose(gt[e], fd(lambda: tab[e], st), rtol=1e-5, atol=1e-9)
    for key, m in [("geo", fl.geo_mlp), ("col", fl.col_mlp)]:
        for l in range(m.n_hidden + 1):
            W = m.W[l] = m.W[l].astype(np.float64)
            b = m.b[l] = m.b[l].astype(np.float64)
            for _ in range(3):
                e = (rng.integers(W.shape[0]), rng.integers(W.shape[1]))

                def st(v, W=W, e=e):
                    W[e] = v
                np.testing.assert_allclose(g[key + "_W"][l][e], fd(lambda: W[e], st), rtol=1e-5, atol=1e-9)
            j = rng.integers(len(b))

            def st(v, b=b, j=j):
                b[j] = v
            np.testing.assert_allclose(g[key + "_b"][l][j], fd(lambda: b[j], st), rtol=1e-5, atol=1e-9)
