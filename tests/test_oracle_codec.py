"""Pins of the oracle's 8-bit min-max grid codec against its definition."""
import numpy as np

import oracle


def test_affine_ramp_codes_exactly():
    # a level holding lo + k * step for k = 0..255 codes to k
    lo, step = -0.75, 0.01
    vals = (lo + step * np.arange(256)).astype(np.float32)
    t = np.tile(vals, 2).reshape(1, 256, 2)
    codes, q, dec = oracle.quantize_grid(t)
    assert q[0, 0] == np.float32(lo)
    assert abs(q[0, 1] - step) < 1e-7
    assert sorted(set(codes.ravel().tolist())) == list(range(256))
    np.testing.assert_allclose(dec, t, atol=1e-6)


def test_extremes_and_round_trip_bound():
    rng = np.random.default_rng(0)
    t = rng.normal(0, 0.3, (3, 4096, 2)).astype(np.float32)
    t[1] = 0.25  # a constant level: step 0, every code 0, decoded exactly
    codes, q, dec = oracle.quantize_grid(t)
    for l in (0, 2):
        assert codes[l].min() == 0 and codes[l].max() == 255
        assert q[l, 0] == t[l].min()
        assert np.abs(dec[l] - t[l]).max() <= 0.5 * q[l, 1] * (1 + 1e-5)
    assert q[1, 1] == 0.0 and codes[1].max() == 0 and np.array_equal(dec[1], t[1].astype(np.float64))
