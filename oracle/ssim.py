"""Plain float64 NumPy / SciPy reference of the SSIM term of Eq. 2 (test
infrastructure; see the package docstring for who may import it).

Eq. 2 adds tau L_S(V, V') to the mapping loss (tau = 0.2, Sec. 4), with L_S
the SSIM loss of Wang et al.  Reading: L_S = 1 - mean SSIM over every pixel
and colour channel, SSIM computed per channel with an 11 x 11 Gaussian window
(sigma 1.5, weights normalised to sum 1), zero padding outside the image
("same"-size maps), C1 = 0.01^2 and C2 = 0.03^2 for images in [0, 1]:

    SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x + s_y + C2)),
    mu_x = G * x,  s_x = G * x^2 - mu_x^2,  s_xy = G * (x y) - mu_x mu_y.

The gradient with respect to the rendered image x follows by the chain
rule through the five local moments:

    dSSIM(p)/dx(q) = G(p - q) [S_mu(p) + S_s(p) (2 x(q) - 2 mu_x(p)) + S_c(p) (y(q) - mu_y(p))],
    S_mu = dSSIM/dmu_x, S_s = dSSIM/ds_x, S_c = dSSIM/ds_xy.
"""

from __future__ import annotations

import numpy as np
from scipy import ndimage

C1 = 0.01 ** 2
C2 = 0.03 ** 2
RADIUS = 5
SIGMA = 1.5


def window_1d() -> np.ndarray:
    k = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-k * k / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def _blur(a: np.ndarray) -> np.ndarray:
    w = np.outer(window_1d(), window_1d())
    return ndimage.correlate(a, w, mode="constant", cval=0.0)


def ssim_maps(x: np.ndarray, y: np.ndarray):
    """Per-channel SSIM map and its partial derivatives for one channel
    (x rendered, y observed; (H, W) arrays)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = _blur(x), _blur(y)
    sx = _blur(x * x) - mx * mx
    sy = _blur(y * y) - my * my
    sxy = _blur(x * y) - mx * my
    a = 2 * mx * my + C1
    b = 2 * sxy + C2
    c = mx * mx + my * my + C1
    d = sx + sy + C2
    S = a * b / (c * d)
    S_mu = 2 * my * b / (c * d) - 2 * mx * S / c
    S_s = -S / d
    S_c = 2 * a / (c * d)
    return S, S_mu, S_s, S_c, mx, my


def _term_magnitude(x, y, S_mu, S_s, S_c, mx, my):
    """sum_p G(p - q) (|S_mu| + 2 |S_s| |x(q) - mu_x(p)| + |S_c| |y(q) - mu_y(p)|)
    for every q, by one shifted copy of the maps per window offset (maps are
    zero outside the image)."""
    H, W = x.shape
    g = window_1d()
    pad = lambda a: np.pad(a, RADIUS)
    Pmu, Ps, Pc, Pmx, Pmy = (pad(a) for a in (S_mu, S_s, S_c, mx, my))
    out = np.zeros_like(x)
    for dy in range(2 * RADIUS + 1):
        for dx in range(2 * RADIUS + 1):
            sl = (slice(dy, dy + H), slice(dx, dx + W))
            out += g[dy] * g[dx] * (np.abs(Pmu[sl]) + 2 * np.abs(Ps[sl]) * np.abs(x - Pmx[sl]) +
                                    np.abs(Pc[sl]) * np.abs(y - Pmy[sl]))
    return out


def ssim_loss(rgb, obs_rgb, w: float = 1.0, magnitude: bool = False):
    """w * L_S and its gradient with respect to rgb ((3, H, W) arrays).
    With magnitude=True also the componentwise magnitude of each gradient
    element, |w|/n sum_p G(p - q) (|S_mu| + 2 |S_s| |x(q) - mu_x| + |S_c|
    |y(q) - mu_y|)(p): the size of the terms its window sum adds."""
    rgb = np.asarray(rgb, np.float64)
    obs = np.asarray(obs_rgb, np.float64)
    n = rgb.size
    total = 0.0
    grad = np.zeros_like(rgb)
    mag = np.zeros_like(rgb)
    for ch in range(rgb.shape[0]):
        x, y = rgb[ch], obs[ch]
        S, S_mu, S_s, S_c, mx, my = ssim_maps(x, y)
        total += S.sum()
        A = S_mu - 2 * mx * S_s - my * S_c
        g = _blur(A) + 2 * x * _blur(S_s) + y * _blur(S_c)   # symmetric window
        grad[ch] = -w / n * g
        if magnitude:
            mag[ch] = abs(w) / n * _term_magnitude(x, y, S_mu, S_s, S_c, mx, my)
    if magnitude:
        return w * (1.0 - total / n), grad, mag
    return w * (1.0 - total / n), grad
