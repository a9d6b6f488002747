"""Pins of the oracle's adaptive density control (3DGS rules the paper keeps)
against hand-built cases and brute-force counts."""
import math

import numpy as np

import oracle


def _case():
    # 6 Gaussians; visible rows for g = 4, 1, 2, 5 (in that order); 0, 3 unseen
    vis = np.array([4, 1, 2, 5], dtype=np.int32)
    alpha = np.array([0.5, 0.5, 0.001, 0.9], dtype=np.float32)       # g=2 below min opacity
    scale = np.array([[0.02, 0.01, 0.01],                            # g=4 large -> split
                      [0.001, 0.002, 0.001],                         # g=1 small -> clone
                      [0.5, 0.5, 0.5],                               # g=2 pruned first
                      [0.001, 0.001, 0.001]], dtype=np.float32)      # g=5 small, low gradient
    accum = np.array([9.0, 0.003, 1.0, 0.0, 0.004, 1e-5], dtype=np.float32)
    count = np.array([0, 3, 1, 0, 2, 1], dtype=np.int32)
    return vis, alpha, scale, accum, count


def test_plan_hand_cases():
    vis, alpha, scale, accum, count = _case()
    act, row, off, total = oracle.densify_plan(6, vis, alpha, scale, accum, count, 2e-4, 0.01, 0.005)
    # g0 unseen (its large accumulated gradient does not matter), g1 clone,
    # g2 prune, g3 unseen, g4 split, g5 keep (1e-5 < 2e-4)
    assert act.tolist() == [0, 2, 1, 0, 3, 0]
    assert row.tolist() == [-1, 1, 2, -1, 0, 3]
    assert off.tolist() == [0, 1, 3, 3, 4, 6, 7] and total == 7


def test_apply_layout_and_split_geometry():
    vis, alpha, scale, accum, count = _case()
    act, row, off, total = oracle.densify_plan(6, vis, alpha, scale, accum, count, 2e-4, 0.01, 0.005)
    rng = np.random.default_rng(3)
    noise = rng.standard_normal((6, 2, 3))
    quat = np.tile([1.0, 0.0, 0.0, 0.0], (4, 1))  # identity rotations
    pos = rng.standard_normal((6, 3))
    new_pos = oracle.densify_apply(act, row, off, scale, quat, noise, math.log(1.6), pos, 2)
    assert new_pos.shape == (7, 3)
    np.testing.assert_array_equal(new_pos[0], pos[0])                   # kept
    np.testing.assert_array_equal(new_pos[1], pos[1])                   # clone original
    np.testing.assert_array_equal(new_pos[2], pos[1])                   # clone copy
    np.testing.assert_array_equal(new_pos[3], pos[3])                   # g2 pruned, g3 kept
    for k in range(2):                                                  # g4 split, identity R
        np.testing.assert_allclose(new_pos[4 + k], pos[4] + scale[0] * noise[4, k], rtol=1e-7)
    np.testing.assert_array_equal(new_pos[6], pos[5])
    # state: zero for the clone copy and both split halves
    m = rng.uniform(1, 2, 6)
    new_m = oracle.densify_apply(act, row, off, scale, quat, noise, math.log(1.6), m, 1)
    assert new_m.tolist() == [m[0], m[1], 0.0, m[3], 0.0, 0.0, m[5]]
    # explicit scale logit lowered by ln 1.6 on the split halves only
    se = rng.uniform(-5, -2, 6)
    new_se = oracle.densify_apply(act, row, off, scale, quat, noise, math.log(1.6), se, 3)
    np.testing.assert_allclose(new_se, [se[0], se[1], se[1], se[3], se[4] - math.log(1.6),
                                        se[4] - math.log(1.6), se[5]])
    # and sigma(x - ln 1.6) ~ sigma(x) / 1.6 for small scales (3DGS's /(0.8 x 2))
    sig = lambda x: 1 / (1 + np.exp(-x))
    assert abs(sig(se[4] - math.log(1.6)) / (sig(se[4]) / 1.6) - 1) < 0.02


def test_split_rotation_is_applied():
    # q = (cos t, 0, 0, sin t): rotation by 2t about z; q and -q give the same
    act = np.array([3], np.uint8)
    row = np.array([0], np.int32)
    off = np.array([0, 2], np.int64)
    scale = np.array([[0.3, 0.1, 0.2]])
    noise = np.array([[[1.0, 0.0, 0.0], [0.0, 1.0, 1.0]]])
    t = 0.25 * math.pi  # 90 degrees about z
    q = np.array([[math.cos(t), 0.0, 0.0, math.sin(t)]])
    p = np.zeros((1, 3))
    a = oracle.densify_apply(act, row, off, scale, q, noise, 0.0, p, 2)
    b = oracle.densify_apply(act, row, off, scale, -q, noise, 0.0, p, 2)
    np.testing.assert_allclose(a, [[0.0, 0.3, 0.0], [-0.1, 0.0, 0.2]], atol=1e-12)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_stats_brute_force():
    rng = np.random.default_rng(5)
    n, nv, W, H = 50, 30, 640, 480
    vis = np.sort(rng.choice(n, nv, replace=False)).astype(np.int32)
    dm = rng.standard_normal((nv, 2)).astype(np.float32) * 1e-4
    nt = rng.integers(0, 3, nv).astype(np.int32)
    acc, cnt = oracle.densify_stats(n, vis, dm, nt, W, H, np.zeros(n), np.zeros(n))
    ref_a, ref_c = np.zeros(n), np.zeros(n, int)
    for i, g in enumerate(vis):
        if nt[i] > 0:
            ref_a[g] += math.hypot(dm[i, 0] * W / 2, dm[i, 1] * H / 2)
            ref_c[g] += 1
    np.testing.assert_allclose(acc, ref_a, rtol=1e-6)
    assert cnt.tolist() == ref_c.tolist()
