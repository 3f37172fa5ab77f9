"""Pins of the FP64 oracle against closed forms, textbook routines, brute
force and invariants (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_25191_gb300 import synth
from tests.scenes import Y00, at_pixel, make_scene, pinhole_views

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "compositing_closed_forms.json")


# ---------------------------------------------------------------------------
# spherical harmonics
# ---------------------------------------------------------------------------

def _random_dirs(n, seed=0):
    d = np.random.default_rng(seed).standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_sh_matches_scipy_condon_shortley():
    """Real SH with the Condon-Shortley phase: Y_lm = sqrt2 Re Y_l^m (m>0),
    sqrt2 Im Y_l^|m| (m<0), Y_l^0 (m=0), with scipy's complex Y_l^m."""
    from scipy.special import sph_harm_y
    for d in _random_dirs(20):
        Y, _ = O.sh_basis(3, d)
        theta = math.acos(np.clip(d[2], -1, 1))
        phi = math.atan2(d[1], d[0])
        for l in range(4):
            for m in range(-l, l + 1):
                c = sph_harm_y(l, abs(m), theta, phi)
                ref = c.real if m == 0 else (math.sqrt(2) * (c.real if m > 0 else c.imag))
                assert abs(Y[l * l + l + m] - ref) < 1e-12


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi: exact for degree <= 6 products
    xs, ws = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for z, w in zip(xs, ws):
        for k in range(nphi):
            phi = 2 * math.pi * k / nphi
            s = math.sqrt(1 - z * z)
            Y, _ = O.sh_basis(3, [s * math.cos(phi), s * math.sin(phi), z])
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_low_orders_closed_form():
    c0, c1 = 0.5 / math.sqrt(math.pi), math.sqrt(3 / (4 * math.pi))
    for x, y, z in _random_dirs(5, 3):
        Y, _ = O.sh_basis(1, [x, y, z])
        assert np.allclose(Y, [c0, -c1 * y, c1 * z, -c1 * x], atol=1e-14)


def test_sh_derivative_matches_finite_difference():
    for d in _random_dirs(5, 4):
        _, dY = O.sh_basis(3, d)
        h = 1e-6
        for j in range(3):
            e = np.zeros(3)
            e[j] = h
            fd = (O.sh_basis(3, d + e)[0] - O.sh_basis(3, d - e)[0]) / (2 * h)
            assert np.abs(fd - dY[:, j]).max() < 1e-7


# ---------------------------------------------------------------------------
# projection
# ---------------------------------------------------------------------------

def test_projection_on_axis_isotropic_closed_form():
    f, z, s = 128.0, 4.0, 0.05
    sc = make_scene([[0, 0, z]], s, 0.5, [[0.5, 0.5, 0.5]])
    vw = pinhole_views(64, 64, f)
    p = O.project_view(sc, vw, 0)
    a = (f * float(np.float32(s)) / z) ** 2 + 0.3
    assert abs(p["cov"][0, 0] - a) < 1e-6 * a and abs(p["cov"][0, 1]) < 1e-9 and abs(p["cov"][0, 2] - a) < 1e-6 * a
    assert np.allclose(p["conic"][0], [1 / a, 0, 1 / a], rtol=1e-6)
    lam = a + math.sqrt(0.1)   # discriminant 0 is floored to 0.1
    assert p["radius"][0] == math.ceil(3 * math.sqrt(lam))
    assert np.allclose(p["xy"][0], [32, 32]) and p["depth"][0] == z


def _quat_rotate(q, v):
    """Hamilton product q v q*, an independent way to rotate by a quaternion."""
    def mul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    q = np.asarray(q, np.float64) / np.linalg.norm(q)
    qc = q * np.array([1, -1, -1, -1])
    return mul(mul(q, np.concatenate([[0.0], v])), qc)[1:]


@pytest.mark.parametrize("rotated_camera", [False, True])
def test_projection_matches_monte_carlo_moments(rotated_camera):
    """Sample 3D points from the Gaussian (rotation by Hamilton products),
    project them with the exact pinhole map, compare the 2D moments with the
    EWA covariance (minus dilation) and the projected mean."""
    rng = np.random.default_rng(7)
    q = np.array([0.8, 0.3, -0.4, 0.33])
    s = np.array([0.012, 0.004, 0.007])
    if rotated_camera:
        vm = synth.look_at((1.0, -0.5, -3.0), target=(0.1, 0.05, 0.2))
        mean = np.array([0.1, 0.05, 0.2])
    else:
        vm = np.concatenate([np.eye(3).reshape(-1), np.zeros(3)])
        mean = np.array([0.15, -0.1, 3.0])
    sc = make_scene([mean], [s], 0.5, [[0.5, 0.5, 0.5]], quats=[q])
    vw = pinhole_views(200, 200, 300.0, viewmat=vm)
    p = O.project_view(sc, vw, 0)
    qf = sc.quats[0].astype(np.float64)
    sf = np.exp(sc.log_scales[0].astype(np.float64))
    cols = np.stack([_quat_rotate(qf, e) for e in np.eye(3)], axis=1)   # rotation matrix columns
    n = 400000
    pts = sc.means[0].astype(np.float64) + (rng.standard_normal((n, 3)) * sf) @ cols.T
    R = vw.viewmats[0, :9].astype(np.float64).reshape(3, 3)
    t = vw.viewmats[0, 9:].astype(np.float64)
    pc = pts @ R.T + t
    u = 300.0 * pc[:, 0] / pc[:, 2] + 100.0
    v = 300.0 * pc[:, 1] / pc[:, 2] + 100.0
    cov = np.cov(np.stack([u, v]))
    ewa = np.array([[p["cov"][0, 0] - 0.3, p["cov"][0, 1]], [p["cov"][0, 1], p["cov"][0, 2] - 0.3]])
    scale = np.abs(ewa).max()
    assert np.abs(cov - ewa).max() < 0.02 * scale
    assert abs(u.mean() - p["xy"][0, 0]) < 0.02 and abs(v.mean() - p["xy"][0, 1]) < 0.02


def test_opacity_aware_extent_bounds_the_alpha_region():
    """Every pixel that gets alpha >= alpha_min lies within the tile extents,
    and the extents are tight: the ellipse o G = alpha_min touches them."""
    sc, vw = _small(n=200, seed=9)
    p = O.project_view(sc, vw, 0)
    ok = p["radius"] > 0
    for g in np.nonzero(ok)[0][:50]:
        A, B, C = p["conic"][g]
        k = 2 * math.log(p["opac"][g] * 255.0)
        # extreme x of the ellipse d^T Q d = k: d = t Q^-1 e_x scaled to the boundary
        cov = np.linalg.inv(np.array([[A, B], [B, C]]))
        ex_true = math.sqrt(k * cov[0, 0])
        assert abs(min(p["radius"][g], ex_true) - p["ext"][g, 0]) < 1e-9 * max(1, ex_true)
        d = cov[:, 0] * math.sqrt(k / cov[0, 0])           # boundary point with the largest |dx|
        alpha = p["opac"][g] * math.exp(-0.5 * d @ np.array([[A, B], [B, C]]) @ d)
        assert abs(alpha - 1 / 255) < 1e-9


def test_transparent_gaussians_are_culled():
    sc = make_scene([[0, 0, 2.0]], 0.05, 0.5 / 255, [[0.5] * 3])
    assert O.project_view(sc, pinhole_views(32, 32, 40.0), 0)["radius"][0] == 0


def test_near_plane_and_nonfinite_culled():
    sc = make_scene([[0, 0, 0.19], [0, 0, 0.21], [0, 0, 3.0]], 0.01, 0.5, [[0.5] * 3] * 3)
    sc.means[2, 0] = np.nan
    p = O.project_view(sc, pinhole_views(64, 64, 100.0, n=3), 0)
    assert p["radius"][0] == 0 and p["radius"][1] > 0 and p["radius"][2] == 0


# ---------------------------------------------------------------------------
# binning
# ---------------------------------------------------------------------------

def test_binning_matches_interval_bruteforce():
    rng = np.random.default_rng(3)
    n, W, H = 400, 100, 70
    x = rng.uniform(-20, 120, n).astype(np.float32)
    y = rng.uniform(-20, 90, n).astype(np.float32)
    r = rng.integers(0, 25, n).astype(np.int32)
    z = rng.uniform(1, 5, n).astype(np.float32)
    z[5] = z[6]            # one exact depth tie: broken by index
    ext = (r[:, None] * rng.uniform(0.2, 1.0, (n, 2))).astype(np.float32)
    for TW, TH in [(16, 16), (8, 8), (32, 16)]:
        ranges, keys, ids = O.bin_view(x, y, r, z, W, H, TW, TH, ext)
        Gx, Gy = O.tile_grid(W, H, TW, TH)
        lo_x, hi_x = x - ext[:, 0], x + ext[:, 0]   # float32 arithmetic
        lo_y, hi_y = y - ext[:, 1], y + ext[:, 1]
        for ty in range(Gy):
            for tx in range(Gx):
                member = (r > 0) & (np.float32(tx * TW) <= hi_x) & (np.float32((tx + 1) * TW) > lo_x) & \
                         (np.float32(ty * TH) <= hi_y) & (np.float32((ty + 1) * TH) > lo_y)
                idx = np.nonzero(member)[0]
                idx = idx[np.lexsort((idx, z[idx]))]
                s, e = ranges[ty * Gx + tx]
                assert np.array_equal(ids[s:e], idx)
                kk = (z[idx].view(np.uint32).astype(np.uint64) << np.uint64(32)) | idx.astype(np.uint64)
                assert np.array_equal(keys[s:e], kk)


# ---------------------------------------------------------------------------
# compositing closed forms
# ---------------------------------------------------------------------------

F, CX = 128.0, 16.0   # pixel centres map to float32-exact world points


def _one_pixel_scene(opacities, depths, colours, scale=0.02):
    means = [at_pixel(10, 12, z, F, CX, CX) for z in depths]
    return make_scene(means, scale, opacities, colours), pinhole_views(32, 32, F, CX, CX, n=len(depths))


@pytest.mark.parametrize("o", [0.3, 0.7, 0.985, 0.995])
def test_single_gaussian_peak_is_opacity_times_colour(o):
    c = [0.8, 0.4, 0.1]
    sc, vw = _one_pixel_scene([o], [2.0], [c])
    img = O.forward(sc, vw)[0]["image"]
    o32 = 1 / (1 + math.exp(-float(sc.opacity_logits[0])))
    rgb = sc.sh[0, 0].astype(np.float64) * Y00 + 0.5
    alpha = min(o32, 0.99)
    assert np.allclose(img[:, 12, 10], alpha * rgb, atol=1e-12)


def test_stacked_transmittance_golden():
    g = json.load(open(GOLDEN))["stacked_three"]
    sc, vw = _one_pixel_scene(g["opacities"], g["depths"][::-1], g["colours"][::-1])  # input order reversed
    out = O.forward(sc, vw, params=O.Params(bg=tuple(g["bg"])))[0]
    assert np.allclose(out["image"][:, 12, 10], g["expected_pixel"], atol=2e-7)
    assert abs(out["T"][12, 10] - g["expected_T"]) < 1e-12
    assert out["n_contrib"][12, 10] == g["expected_n_contrib"]


def test_early_stop_golden():
    g = json.load(open(GOLDEN))["early_stop"]
    depths = [2.0 + 0.05 * k for k in range(g["count"])]
    sc, vw = _one_pixel_scene([g["opacity"]] * g["count"], depths, [[0.5, 0.5, 0.5]] * g["count"])
    out = O.forward(sc, vw)[0]
    assert out["n_contrib"][12, 10] == g["expected_n_contrib"]
    assert abs(out["T"][12, 10] - g["expected_T"]) < 1e-9


@pytest.mark.parametrize("side,expect", [(1 + 1e-3, True), (1 - 1e-3, False)])
def test_alpha_cutoff_toggles(side, expect):
    sc, vw = _one_pixel_scene([side / 255.0], [2.0], [[1.0, 1.0, 1.0]])
    img = O.forward(sc, vw)[0]["image"]
    assert (img[0, 12, 10] > 0) == expect


# ---------------------------------------------------------------------------
# brute force and invariants on the synthetic small scene
# ---------------------------------------------------------------------------

def _small(n=300, W=40, H=36, seed=2):
    sc = synth.uniform_box_scene(seed, n, lo=(-0.6, -0.6, 2.0), hi=(0.6, 0.6, 4.0), sh_degree=1)
    vw = synth._views(np.concatenate([np.eye(3).reshape(-1), np.zeros(3)]), 60.0, W, H, 0, n)
    return sc, vw


def _bruteforce_image(proj, W, H, TW, TH, prm):
    """Per pixel, all listed Gaussians (square tile rectangle by float32
    interval intersection) passing the square gate, sorted by (float32 depth,
    index), composited directly."""
    n = proj["xy"].shape[0]
    xf = proj["xy"][:, 0].astype(np.float32)
    yf = proj["xy"][:, 1].astype(np.float32)
    zf = proj["depth"].astype(np.float32)
    r = proj["radius"]
    order = np.lexsort((np.arange(n), zf))
    img = np.zeros((3, H, W))
    for py in range(H):
        for px in range(W):
            tx, ty = px // TW, py // TH
            T = 1.0
            col = np.zeros(3)
            for g in order:
                if r[g] <= 0:
                    continue
                rf = np.float32(r[g])
                if not (np.float32(tx * TW) <= xf[g] + rf and np.float32((tx + 1) * TW) > xf[g] - rf and
                        np.float32(ty * TH) <= yf[g] + rf and np.float32((ty + 1) * TH) > yf[g] - rf):
                    continue
                dx, dy = px + 0.5 - proj["xy"][g, 0], py + 0.5 - proj["xy"][g, 1]
                if abs(dx) > r[g] or abs(dy) > r[g]:
                    continue
                A, B, C = proj["conic"][g]
                pw = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
                if pw > 0:
                    continue
                a = min(prm.alpha_max, proj["opac"][g] * math.exp(pw))
                if a < prm.alpha_min:
                    continue
                if T * (1 - a) < prm.t_min:
                    break
                col += proj["rgb"][g] * a * T
                T *= 1 - a
            img[:, py, px] = col + T * np.asarray(prm.bg)
    return img


def test_oracle_render_equals_bruteforce():
    sc, vw = _small()
    prm = O.Params(bg=(0.2, 0.1, 0.05))
    proj = O.project_view(sc, vw, 0, prm)
    for TW, TH in [(16, 16), (8, 8)]:
        bins = O.bin_view(proj["xy"][:, 0], proj["xy"][:, 1], proj["radius"], proj["depth"], 40, 36, TW, TH)   # square rectangles
        out = O.render_view(proj, 40, 36, TW, TH, prm, bins)
        ref = _bruteforce_image(proj, 40, 36, TW, TH, prm)
        assert np.abs(out["image"] - ref).max() < 1e-12
        # lists bounded by the opacity-aware extents give the same image
        assert (proj["ext"][proj["radius"] > 0] < proj["radius"][proj["radius"] > 0, None] - 0.5).any()
        tight = O.forward(sc, vw, TW, TH, prm)[0]["image"]
        assert np.abs(tight - ref).max() < 1e-12


def test_permutation_invariance():
    sc, vw = _small(seed=5)
    assert len(np.unique(sc.means[:, 2])) == sc.n
    a = O.forward(sc, vw)[0]["image"]
    perm = np.random.default_rng(0).permutation(sc.n)
    b = O.forward(sc.permuted(perm), vw)[0]["image"]
    assert np.array_equal(a, b)


def test_tile_size_invariance_with_pixel_gate():
    sc, vw = _small(seed=6)
    imgs = [O.forward(sc, vw, TW, TH)[0]["image"] for TW, TH in [(16, 16), (8, 8), (32, 8), (4, 32)]]
    for im in imgs[1:]:
        assert np.array_equal(imgs[0], im)


def test_translation_invariance():
    sc, vw = _small(seed=8)
    a = O.forward(sc, vw)[0]["image"]
    shift = np.array([0.25, -0.5, 0.125], np.float32)   # exact in float32
    sc2 = sc.subset(slice(None))
    sc2.means = sc.means + shift
    vw2 = vw.select([0])
    vw2.viewmats[0, 9:] = -shift                        # t' = t - R shift, R = I
    b = O.forward(sc2, vw2)[0]["image"]
    assert np.abs(a - b).max() < 1e-6


def test_batched_views_equal_single_views():
    sc, vw = synth.orbit_views(0, 2000, 3, 48, 40, 60.0)
    full = O.forward(sc, vw)
    for v in range(3):
        one = O.forward(sc, vw.select([v]))[0]
        assert np.array_equal(full[v]["image"], one["image"])
