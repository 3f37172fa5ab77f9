"""FP64 oracle of the photometric loss with D-SSIM (Section 3.1).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline); shares no code
with the CUDA library.

Section 3.1 trains with a weighted sum of an L1 term and a D-SSIM term; the
weight and the SSIM settings come from the cited 3DGS training:
    L = (1 - lambda) * mean|x - y| + lambda * (1 - mean SSIM(x, y)),
    lambda = 0.2,
with SSIM (Wang et al. 2004) on each colour channel of each view, local
statistics taken with an 11x11 Gaussian window (sigma = 1.5, normalised to
sum 1) as a 'same'-size correlation with zero padding at the image border:
    mu_x = G*x, mu_y = G*y, s_xx = G*(x^2) - mu_x^2, s_yy = G*(y^2) - mu_y^2,
    s_xy = G*(xy) - mu_x mu_y,
    S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),
    C1 = 0.01^2, C2 = 0.03^2 (dynamic range 1),
and the mean taken over every pixel and channel of every view (like the L1
mean). The gradient with respect to the rendered image x follows from
writing S through (mu_x, A = G*(x^2), B = G*(xy)):
    dS/dmu_x = S (2 mu_y / l1 - 2 mu_y / l2 - 2 mu_x / d1 + 2 mu_x / d2),
    dS/dA = -S / d2,  dS/dB = 2 S / l2,
(l1, l2 the numerator factors, d1, d2 the denominator factors) and
    dmean S / dx = G (x) a + 2 x (G (x) b) + y (G (x) c)
with a, b, c those three derivatives divided by the count and (x) the
adjoint (the same zero-padded correlation, the window being symmetric).
Pinned in tests/test_oracle_ssim.py: identical images (SSIM 1, gradient 0),
the closed form of constant images, a per-pixel brute-force windowed sum
with explicit zero padding, central differences, symmetry.
"""
import numpy as np
from scipy.signal import correlate2d

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA = 0.2


def gaussian_1d(size=WINDOW, sigma=SIGMA):
    k = np.arange(size) - (size - 1) / 2.0
    g = np.exp(-k * k / (2.0 * sigma * sigma))
    return g / g.sum()


def window(size=WINDOW, sigma=SIGMA):
    g = gaussian_1d(size, sigma)
    return np.outer(g, g)


def _filt(img, win):
    return correlate2d(img, win, mode="same", boundary="fill", fillvalue=0.0)


def ssim_map(x, y, win=None):
    """Per-pixel SSIM of two [H,W] FP64 images."""
    win = window() if win is None else win
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = _filt(x, win), _filt(y, win)
    sxx = _filt(x * x, win) - mx * mx
    syy = _filt(y * y, win) - my * my
    sxy = _filt(x * y, win) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim_terms(x, y, scale, win=None):
    """(sum of S over the image, d(scale * sum S)/dx) for one [H,W] channel."""
    win = window() if win is None else win
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = _filt(x, win), _filt(y, win)
    sxx = _filt(x * x, win) - mx * mx
    syy = _filt(y * y, win) - my * my
    sxy = _filt(x * y, win) - mx * my
    l1 = 2 * mx * my + C1
    l2 = 2 * sxy + C2
    d1 = mx * mx + my * my + C1
    d2 = sxx + syy + C2
    S = (l1 * l2) / (d1 * d2)
    a = scale * S * (2 * my / l1 - 2 * my / l2 - 2 * mx / d1 + 2 * mx / d2)
    b = scale * (-S / d2)
    c = scale * (2 * S / l2)
    grad = _filt(a, win) + 2 * x * _filt(b, win) + y * _filt(c, win)
    return float(S.sum()), grad


def l1_dssim(images, targets, lam=LAMBDA):
    """images, targets: lists of [3,H,W] views. Returns (total, l1, dssim,
    gradients) with the means over all values of all views."""
    n = sum(np.asarray(im).size for im in images)
    l1 = 0.0
    s = 0.0
    grads = []
    for im, tg in zip(images, targets):
        im = np.asarray(im, np.float64)
        tg = np.asarray(tg, np.float64)
        d = im - tg
        l1 += float(np.abs(d).sum())
        g = (1 - lam) * np.sign(d) / n
        for ch in range(im.shape[0]):
            sc, gs = ssim_terms(im[ch], tg[ch], 1.0 / n)
            s += sc
            g[ch] -= lam * gs
        grads.append(g)
    l1 /= n
    dssim = 1.0 - s / n
    return (1 - lam) * l1 + lam * dssim, l1, dssim, grads
