"""Pins of the FP64 L1 + D-SSIM oracle (Section 3.1 loss)."""
import numpy as np

from oracle import ssim as OS


def test_window_is_a_normalised_sampled_gaussian():
    g = OS.gaussian_1d()
    assert abs(g.sum() - 1) < 1e-15 and np.allclose(g, g[::-1])
    assert np.allclose(g[6:] / g[5:-1], np.exp(-(2 * np.arange(5) + 1) / (2 * 1.5 ** 2)))
    assert OS.window().shape == (11, 11) and abs(OS.window().sum() - 1) < 1e-14


def test_identical_images_have_ssim_one_and_zero_gradient():
    rng = np.random.default_rng(0)
    x = rng.random((3, 23, 31))
    total, l1, dssim, g = OS.l1_dssim([x], [x.copy()])
    assert abs(dssim) < 1e-12 and l1 == 0 and abs(total) < 1e-12
    assert np.abs(g[0]).max() < 1e-12


def test_constant_images_closed_form_in_the_interior():
    a, b = 0.3, 0.7
    S = OS.ssim_map(np.full((30, 30), a), np.full((30, 30), b))
    ref = (2 * a * b + OS.C1) / (a * a + b * b + OS.C1)
    assert np.allclose(S[5:-5, 5:-5], ref, rtol=1e-12)


def _brute_map(x, y):
    """Per-pixel weighted sums over the 11x11 neighbourhood, pixels outside
    the image counted as 0."""
    H, W = x.shape
    w = OS.window()
    out = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            sx = sy = sxx = syy = sxy = 0.0
            for di in range(-5, 6):
                for dj in range(-5, 6):
                    u, v = i + di, j + dj
                    if 0 <= u < H and 0 <= v < W:
                        k = w[di + 5, dj + 5]
                        sx += k * x[u, v]
                        sy += k * y[u, v]
                        sxx += k * x[u, v] ** 2
                        syy += k * y[u, v] ** 2
                        sxy += k * x[u, v] * y[u, v]
            vx, vy, cxy = sxx - sx * sx, syy - sy * sy, sxy - sx * sy
            out[i, j] = ((2 * sx * sy + OS.C1) * (2 * cxy + OS.C2)) / ((sx * sx + sy * sy + OS.C1) * (vx + vy + OS.C2))
    return out


def test_map_against_brute_force_windowed_sums():
    rng = np.random.default_rng(1)
    x, y = rng.random((13, 17)), rng.random((13, 17))
    ref = _brute_map(x, y)
    assert np.allclose(OS.ssim_map(x, y), ref, rtol=1e-12, atol=1e-13)
    assert abs(OS.ssim_terms(x, y, 1.0)[0] - ref.sum()) < 1e-11


def test_symmetry():
    rng = np.random.default_rng(2)
    x, y = rng.random((15, 12)), rng.random((15, 12))
    assert np.allclose(OS.ssim_map(x, y), OS.ssim_map(y, x), rtol=1e-13)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    x = rng.random((3, 9, 14))
    y = np.clip(x + 0.2 * rng.standard_normal(x.shape), 0, 1)
    x2 = rng.random((3, 7, 5))
    y2 = rng.random((3, 7, 5))
    total, l1, dssim, g = OS.l1_dssim([x, x2], [y, y2])
    h = 1e-6
    for v, (im, other) in enumerate(((x, x2), (x2, x))):
        for idx in list(np.ndindex(im.shape))[::3]:
            a = im.copy()
            a[idx] += h
            Lp = OS.l1_dssim([a, other] if v == 0 else [other, a], [y, y2])[0]
            a[idx] -= 2 * h
            Lm = OS.l1_dssim([a, other] if v == 0 else [other, a], [y, y2])[0]
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[v][idx]) <= 1e-6 * (1 + abs(fd)) + 1e-9, (v, idx, fd, g[v][idx])


def test_l1_term_and_weighting():
    x = np.zeros((3, 4, 4))
    y = np.full((3, 4, 4), 0.5)
    total, l1, dssim, g = OS.l1_dssim([x], [y], lam=0.0)
    assert l1 == 0.5 and total == 0.5
    assert np.allclose(g[0], -1.0 / x.size)
    total2, _, dssim2, _ = OS.l1_dssim([x], [y], lam=1.0)
    assert total2 == dssim2
