"""Pins of the SSIM reference (oracle/ssim.py): identity, closed forms on
constant and linear images, the window itself, finite differences."""

import numpy as np
import pytest

from oracle import ssim as os_


def test_window():
    g = os_.window_1d()
    assert g.size == 11 and g.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(g[6] / g[5], np.exp(-1 / 4.5), rtol=1e-14)
    np.testing.assert_allclose(g[10] / g[5], np.exp(-25 / 4.5), rtol=1e-14)
    np.testing.assert_array_equal(g, g[::-1])


def test_identical_images():
    rng = np.random.default_rng(0)
    x = rng.random((3, 20, 17))
    L, g = os_.ssim_loss(x, x, 0.2)
    assert abs(L) < 1e-14 and np.abs(g).max() < 1e-14


def _interior(a):
    return a[5:-5, 5:-5]


@pytest.mark.parametrize("a, b", [(0.3, 0.3), (0.2, 0.7), (0.9, 0.05)])
def test_constant_images(a, b):
    """Interior: no variance, so SSIM = (2ab + C1) / (a^2 + b^2 + C1)."""
    S = os_.ssim_maps(np.full((16, 16), a), np.full((16, 16), b))[0]
    np.testing.assert_allclose(_interior(S), (2 * a * b + os_.C1) / (a * a + b * b + os_.C1),
                               rtol=1e-11)     # variances are E[x^2] - mu^2 ~ 1e-17, not 0


def test_linear_ramp_shift_and_scale():
    """x = 0.02 u + 0.3: in the interior the symmetric window leaves the mean
    at x and the variance at 0.02^2 sum g(k) k^2.  A shifted copy y = x + c
    has the same variances and covariance (structure term 1); a scaled copy
    y = s x has s and s^2 times them."""
    u = np.arange(24, dtype=np.float64)
    x = np.tile(0.02 * u + 0.3, (24, 1))
    g = os_.window_1d()
    var = 0.02 ** 2 * np.sum(g * np.arange(-5, 6) ** 2)
    c = 0.1
    S = os_.ssim_maps(x, x + c)[0]
    xi = _interior(x)
    np.testing.assert_allclose(_interior(S), (2 * xi * (xi + c) + os_.C1) /
                               (xi * xi + (xi + c) ** 2 + os_.C1), rtol=1e-12)
    s = 1.5
    S = os_.ssim_maps(x, s * x)[0]
    lum = (2 * s * xi * xi + os_.C1) / ((1 + s * s) * xi * xi + os_.C1)
    st = (2 * s * var + os_.C2) / ((1 + s * s) * var + os_.C2)
    np.testing.assert_allclose(_interior(S), lum * st, rtol=1e-10)


def test_gradient_is_finite_difference():
    rng = np.random.default_rng(1)
    x = rng.random((3, 13, 15))
    y = np.clip(x + 0.2 * rng.normal(size=x.shape), 0, 1)
    L, g = os_.ssim_loss(x, y, 0.2)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 6, 7), (2, 12, 14), (0, 3, 11), (2, 9, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (os_.ssim_loss(xp, y, 0.2)[0] - os_.ssim_loss(xm, y, 0.2)[0]) / (2 * h)
        assert fd == pytest.approx(g[idx], rel=1e-6, abs=1e-12)
