"""Pins of the oracle's Adam step against closed forms of the published
algorithm (Kingma & Ba 2015, Algorithm 1)."""
import numpy as np

import oracle


def test_first_step_closed_form():
    # t = 1 from zero moments: m_hat = g, v_hat = g^2, so the step is
    # lr * g / (|g| + eps) whatever beta1, beta2 are
    rng = np.random.default_rng(0)
    p0, g = rng.standard_normal(1000), rng.standard_normal(1000) * 1e-3
    for b1, b2 in [(0.9, 0.999), (0.5, 0.99), (0.0, 0.0)]:
        p, m, v = oracle.adam_step(p0, g, np.zeros(1000), np.zeros(1000), 0.01, b1, b2, 1e-8, 1)
        np.testing.assert_allclose(p, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(m, (1 - b1) * g, rtol=1e-12)
        np.testing.assert_allclose(v, (1 - b2) * g * g, rtol=1e-12)


def test_constant_gradient_moves_linearly():
    # a constant gradient gives m_hat = g and v_hat = g^2 at every step:
    # after t steps p = p0 - t lr g / (|g| + eps)
    g = np.array([0.5, -2.0, 3e-4])
    p, m, v = np.array([1.0, 2.0, 3.0]), np.zeros(3), np.zeros(3)
    for t in range(1, 51):
        p, m, v = oracle.adam_step(p, g, m, v, 1e-3, 0.9, 0.999, 1e-15, t)
    np.testing.assert_allclose(p, np.array([1.0, 2.0, 3.0]) - 50 * 1e-3 * np.sign(g), rtol=1e-9)


def test_zero_gradient_decays_moments_and_grad_scale():
    p, m, v = oracle.adam_step([1.0], [0.0], [0.2], [0.04], 0.1, 0.9, 0.99, 1e-15, 3)
    assert m[0] == 0.9 * 0.2 and v[0] == 0.99 * 0.04
    mh, vh = m[0] / (1 - 0.9 ** 3), v[0] / (1 - 0.99 ** 3)
    assert abs(p[0] - (1.0 - 0.1 * mh / (np.sqrt(vh) + 1e-15))) < 1e-15
    # grad_scale multiplies the gradient before both moments
    a = oracle.adam_step([0.0], [4.0], [0.0], [0.0], 1.0, 0.9, 0.99, 1e-15, 2, grad_scale=0.25)
    b = oracle.adam_step([0.0], [1.0], [0.0], [0.0], 1.0, 0.9, 0.99, 1e-15, 2)
    assert np.allclose(a, b, rtol=0, atol=0)
