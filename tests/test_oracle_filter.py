"""Pins of the oracle's V2LF low-pass plane filter (Sec. 4.5) against
properties that fix a separable normalised Gaussian with zero padding."""
import numpy as np


def test_weights_are_a_normalised_gaussian(orc):
    for sigma, r in ((0.5, 2), (1.0, 3), (2.3, 7)):
        w = orc.filter_weights(sigma, r)
        i = np.arange(-r, r + 1)
        g = np.exp(-i * i / (2 * sigma * sigma))
        assert abs(w.sum() - 1.0) < 1e-15
        assert np.allclose(w, g / g.sum(), rtol=0, atol=1e-16)
        assert np.allclose(w, w[::-1], rtol=0, atol=0)


def test_impulse_response_is_the_outer_product(orc):
    sigma, r = 1.3, 4
    p = np.zeros((1, 21, 23, 4))
    p[0, 10, 11, :] = [1.0, 0.5, 0.25, 2.0]
    out = orc.filter_planes(p, sigma, r)
    w = orc.filter_weights(sigma, r)
    k2 = np.outer(w, w)
    for c, a in enumerate([1.0, 0.5, 0.25, 2.0]):
        want = np.zeros((21, 23))
        want[10 - r:10 + r + 1, 11 - r:11 + r + 1] = a * k2
        assert np.abs(out[0, :, :, c] - want).max() < 1e-15


def test_constant_plane_interior_and_border(orc):
    # weights sum to one: a constant plane is unchanged away from the border;
    # on the border zero padding drops exactly the weights outside the plane
    sigma, r = 0.9, 3
    p = np.full((2, 12, 15, 4), 0.7)
    out = orc.filter_planes(p, sigma, r)
    assert np.abs(out[:, r:-r, r:-r, :] - 0.7).max() < 1e-14
    w = orc.filter_weights(sigma, r)
    edge = 0.7 * w[r:].sum() * 1.0          # corner pixel (0, 0): rows and columns each keep w[r:]
    assert abs(out[0, 0, 0, 0] - 0.7 * w[r:].sum() * w[r:].sum()) < 1e-15
    assert abs(out[0, 0, 7, 0] - edge) < 1e-15


def test_filter_is_linear_and_separable(orc):
    rng = np.random.default_rng(3)
    a = rng.random((1, 9, 11, 4))
    b = rng.random((1, 9, 11, 4))
    fa, fb = orc.filter_planes(a, 1.1, 3), orc.filter_planes(b, 1.1, 3)
    assert np.abs(orc.filter_planes(2 * a + b, 1.1, 3) - (2 * fa + fb)).max() < 1e-14
    # brute-force 2D convolution with the outer-product kernel
    w = orc.filter_weights(1.1, 3)
    k2 = np.outer(w, w)
    want = np.zeros_like(a)
    for y in range(9):
        for x in range(11):
            for dy in range(-3, 4):
                for dx in range(-3, 4):
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < 9 and 0 <= xx < 11:
                        want[0, y, x] += k2[dy + 3, dx + 3] * a[0, yy, xx]
    assert np.abs(fa - want).max() < 1e-14
