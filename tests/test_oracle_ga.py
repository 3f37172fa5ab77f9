"""Pins of the FP64 global-alignment oracle (Section 3.3, Eqs. 2-4) against
what the geometry and the definitions fix, independently of its formulas."""
import statistics

import numpy as np
import pytest

from oracle import ga
from paper_2509_25191_gb300 import synth


def _project(P, intr, vm):
    """Independent pinhole projection x = K (R X + t) / z."""
    R, t = vm[:9].reshape(3, 3), vm[9:]
    Xc = P @ R.T + t
    return np.stack([intr[0] * Xc[:, 0] / Xc[:, 2] + intr[2], intr[1] * Xc[:, 1] / Xc[:, 2] + intr[3]], 1)


def _ortho(vms):
    """float64 copies with each R replaced by the nearest rotation (the
    epipolar geometry assumes R^-1 = R^T, which float32 storage breaks at
    1e-7)."""
    out = np.array(vms, np.float64).reshape(-1, 12)
    for v in out:
        U, _, Vt = np.linalg.svd(v[:9].reshape(3, 3))
        v[:9] = (U @ Vt).reshape(-1)
    return out


def _cams(n=6, seed=0):
    tv, ti, iv, ii = synth.ga_cameras(seed, n_views=n, width=640, height=480, focal=500.0)
    return _ortho(tv), ti.astype(np.float64), _ortho(iv), ii.astype(np.float64)


def _center(vm):
    return -vm[:9].reshape(3, 3).T @ vm[9:]


def test_exact_matches_have_zero_distance():
    # float64 rotations: the epipolar constraint holds exactly only for
    # orthonormal R, which float32 storage perturbs at 1e-7
    tv = synth.hemisphere_viewmats(6).reshape(6, 12)
    ti = np.tile([500.0, 480.0, 320.0, 240.0], (6, 1))
    P = synth.ga_points(3, 200, 1.5)
    for i, j in [(0, 1), (2, 5), (4, 3)]:
        F = ga.fundamental(ti[i], ti[j], tv[i], tv[j])
        e = ga.epipolar_distance(F, _project(P, ti[i], tv[i]), _project(P, ti[j], tv[j]))
        assert e.max() < 1e-9, e.max()


def test_fundamental_has_rank_two_and_the_epipoles_as_null_vectors():
    tv = synth.jitter_viewmats(synth.hemisphere_viewmats(6), 3, 5.0, 0.2)      # float64, orthonormal
    ti = np.tile([500.0, 480.0, 320.0, 240.0], (6, 1))
    for i, j in [(0, 1), (1, 4)]:
        F = ga.fundamental(ti[i], ti[j], tv[i], tv[j])
        sv = np.linalg.svd(F, compute_uv=False)
        assert sv[2] < 1e-12 * sv[0]
        # epipole in image i = image of camera j's centre, and vice versa
        ei = np.append(_project(_center(tv[j])[None], ti[i], tv[i])[0], 1.0)
        ej = np.append(_project(_center(tv[i])[None], ti[j], tv[j])[0], 1.0)
        assert np.abs(F @ ei).max() < 1e-12 * np.abs(F).max() * np.abs(ei).max()
        assert np.abs(ej @ F).max() < 1e-12 * np.abs(F).max() * np.abs(ej).max()
        # the orientation matters: F^T does not annihilate e_i
        assert np.abs(F.T @ ei).max() > 1e-6 * np.abs(F).max() * np.abs(ei).max()


def test_distance_equals_the_point_to_line_distance_of_the_projected_ray():
    """The epipolar line of x is the image, in camera j, of the ray from
    camera i's centre through x; built from two projected ray points."""
    _, _, iv, ii = _cams()
    rng = np.random.default_rng(5)
    i, j = 0, 2
    x = rng.uniform([0, 0], [640, 480], (50, 2))
    xp = rng.uniform([0, 0], [640, 480], (50, 2))
    F = ga.fundamental(ii[i], ii[j], iv[i], iv[j])
    e = ga.epipolar_distance(F, x, xp)
    Ri = iv[i, :9].reshape(3, 3)
    Ci = _center(iv[i])
    rays = np.stack([(x[:, 0] - ii[i, 2]) / ii[i, 0], (x[:, 1] - ii[i, 3]) / ii[i, 1], np.ones(50)], 1) @ Ri
    p1 = _project(Ci + 2.0 * rays, ii[j], iv[j])
    p2 = _project(Ci + 6.0 * rays, ii[j], iv[j])
    d = p2 - p1
    ref = np.abs(d[:, 0] * (xp[:, 1] - p1[:, 1]) - d[:, 1] * (xp[:, 0] - p1[:, 0])) / np.hypot(d[:, 0], d[:, 1])
    assert np.allclose(e, ref, rtol=1e-9, atol=1e-9)


def _problem(n=5, per_pair=30, seed=0):
    tv, ti, iv, ii = _cams(n, seed)
    pairs = np.array([(0, 1), (0, 2), (1, 3), (2, 4), (3, 4), (1, 2)], np.int32)
    M = synth.ga_matches(seed, synth.ga_points(seed, 400, 1.5), ti, tv, pairs, 640, 480, per_pair, 0.8, 0.2)
    w = np.random.default_rng(seed).uniform(0.2, 1.5, len(M.matches))
    return ii, iv, pairs, M, w


def test_gradients_match_central_differences():
    intr, vms, pairs, M, w = _problem()
    L, d_intr, d_vm = ga.loss_and_grads(intr, vms, pairs, M.offsets, M.matches, w)
    h = 1e-6
    for arr, grad, scale in ((intr, d_intr, 100.0), (vms, d_vm, 1.0)):
        for idx in np.ndindex(arr.shape):
            a = arr.copy()
            a[idx] += h * scale
            Lp = ga.loss_and_grads(a if arr is intr else intr, a if arr is vms else vms, pairs, M.offsets,
                                   M.matches, w)[0]
            a[idx] -= 2 * h * scale
            Lm = ga.loss_and_grads(a if arr is intr else intr, a if arr is vms else vms, pairs, M.offsets,
                                   M.matches, w)[0]
            fd = (Lp - Lm) / (2 * h * scale)
            assert abs(fd - grad[idx]) <= 1e-6 * (1 + abs(fd)), (idx, fd, grad[idx])
    assert np.abs(d_vm).max() > 1e-3 and np.abs(d_intr).max() > 1e-6


def _axis_rot(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = ga.skew(a)
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def test_loss_is_invariant_to_the_similarity_gauge_and_its_gradient_orthogonal_to_it():
    intr, vms, pairs, M, w = _problem(seed=1)
    L, d_intr, d_vm = ga.loss_and_grads(intr, vms, pairs, M.offsets, M.matches, w)
    Q = _axis_rot([0.3, -1.0, 0.5], 0.4)
    c = np.array([0.7, -0.2, 1.1])
    s = 1.7
    moved = vms.copy()
    for n in range(len(vms)):
        R, t = vms[n, :9].reshape(3, 3), vms[n, 9:]
        # world point Y = s Q X + c: camera coordinates scale by s
        moved[n, :9] = (R @ Q.T).reshape(-1)
        moved[n, 9:] = s * t - R @ Q.T @ c
    L2 = ga.loss_and_grads(intr, moved, pairs, M.offsets, M.matches, w)[0]
    assert abs(L2 - L) <= 1e-10 * L
    G_R, G_t = d_vm[:, :9].reshape(-1, 3, 3), d_vm[:, 9:]
    R = vms[:, :9].reshape(-1, 3, 3)
    t = vms[:, 9:]
    scale = np.abs(d_vm).max() * 10
    assert abs(np.sum(G_t * t)) < 1e-9 * scale                          # global scale
    for cc in np.eye(3):
        assert abs(np.sum(G_t * (R @ cc))) < 1e-9 * scale               # world translation
        Om = ga.skew(cc)
        assert abs(np.sum(G_R * (R @ Om))) < 1e-9 * scale               # world rotation
    assert np.abs(G_t).max() > 1e-4


def test_histogram_weights_against_numpy_density():
    rng = np.random.default_rng(2)
    e = np.abs(rng.standard_cauchy(5000)).astype(np.float32)
    e = np.minimum(e, np.float32(40.0))
    B = 64
    w, counts = ga.pdf_weights(e, B, 0.5)
    dens, edges = np.histogram(e.astype(np.float64), bins=B, range=(0.0, float(e.max())), density=True)
    idx = np.clip(np.searchsorted(edges, e.astype(np.float64), side="right") - 1, 0, B - 1)
    away = np.abs(e[:, None] - edges[None, 1:-1]).min(1) > 1e-4 * float(e.max())
    f = dens[idx]
    ref = (f / f.mean()) ** 0.5
    assert away.sum() > 4900
    assert np.allclose(w[away], ref[away], rtol=1e-3)
    assert counts.sum() == len(e)


def test_histogram_weights_closed_forms():
    # one value per bin: flat density, every weight 1
    B = 10
    e = (np.arange(B, dtype=np.float32) + 0.5) * np.float32(0.3)
    w, _ = ga.pdf_weights(e, B, 0.5)
    assert np.allclose(w, 1.0, rtol=1e-12)
    # 75 % in the first bin, 25 % in the last: densities in ratio 3:1, mean
    # density 0.75*3 + 0.25*1 = 2.5 (units of the last bin's density)
    e = np.array([0.1] * 6 + [9.9, 10.0], np.float32)
    w, counts = ga.pdf_weights(e, B, 0.5)
    assert counts[0] == 6 and counts[-1] == 2
    assert np.allclose(w[:6], np.sqrt(3 / 2.5)) and np.allclose(w[6:], np.sqrt(1 / 2.5))
    # alpha = 1: the plain density ratio
    w1, _ = ga.pdf_weights(e, B, 1.0)
    assert np.allclose(w1[:6], 3 / 2.5) and np.allclose(w1[6:], 1 / 2.5)
    # all distances equal zero: one bin, weight 1
    w0, c0 = ga.pdf_weights(np.zeros(7, np.float32), B, 0.5)
    assert np.allclose(w0, 1.0) and c0[0] == 7


def test_median_against_its_definition():
    rng = np.random.default_rng(4)
    for K in (1, 2, 7, 10, 101):
        e = rng.exponential(3.0, K).astype(np.float32)
        lo, hi, med = ga.median_order_stats(e)
        assert med == pytest.approx(statistics.median([float(v) for v in e]), rel=0, abs=0)
        assert np.sum(e < lo) <= (K - 1) // 2 <= np.sum(e <= lo) - 1
        assert np.sum(e < hi) <= K // 2 <= np.sum(e <= hi) - 1


def test_learning_rate_rule():
    assert ga.lr_rule(0.3) == 5e-4
    assert ga.lr_rule(2.4999) == 5e-4
    assert ga.lr_rule(2.5) == 1e-3
    assert ga.lr_rule(7.5) == 1e-3
    assert ga.lr_rule(7.5001) == 1e-2
    assert ga.lr_rule(300.0) == 1e-2


def test_pair_selection_by_viewing_angle():
    # orbit cameras 12 degrees apart: neighbours at 12 and 24 degrees pass,
    # 36 degrees does not
    n = 30
    mats = synth.orbit_viewmats(n, 5.0)
    mats = np.asarray(mats, np.float32).reshape(n, 12)
    pairs = ga.select_pairs(mats, 30.0)
    ref = [(i, j) for i in range(n) for j in range(i + 1, n) if min(j - i, n - (j - i)) <= 2]
    assert [tuple(p) for p in pairs] == ref
    # random hemisphere cameras: brute force in float64 away from the threshold
    tv, _, iv, _ = synth.ga_cameras(0, 120, 640, 480, 500.0)
    pairs = {tuple(p) for p in ga.select_pairs(iv, 30.0)}
    d = iv[:, 6:9].astype(np.float64)
    for i in range(120):
        for j in range(i + 1, 120):
            ang = np.degrees(np.arccos(np.clip(d[i] @ d[j] / np.linalg.norm(d[i]) / np.linalg.norm(d[j]), -1, 1)))
            if abs(ang - 30.0) > 1e-3:
                assert ((i, j) in pairs) == (ang < 30.0), (i, j, ang)


def test_residual_identity_and_orthonormality():
    _, _, iv, ii = _cams(4)
    ident = np.tile([1.0, 0, 0, 0, 1.0, 0, 0, 0, 0, 0], (4, 1))
    intr, vm = ga.apply_residuals(ii, iv, ident)
    assert np.allclose(vm, iv, atol=1e-15) and np.allclose(intr, ii, atol=1e-12)
    rng = np.random.default_rng(1)
    for _ in range(5):
        R = ga.rotation_6d(rng.standard_normal(6))
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-13) and abs(np.linalg.det(R) - 1) < 1e-13
    # a rotation about z by theta has 6D representation (cos, sin, 0, -sin, cos, 0)
    th = 0.3
    R = ga.rotation_6d([np.cos(th), np.sin(th), 0, -np.sin(th), np.cos(th), 0])
    assert np.allclose(R, _axis_rot([0, 0, 1], th), atol=1e-15)


def test_residual_vjp_matches_central_differences():
    intr0, vm0, pairs, M, w = _problem(seed=2)
    rng = np.random.default_rng(3)
    res = np.tile([1.0, 0, 0, 0, 1.0, 0, 0, 0, 0, 0], (len(vm0), 1)) + 0.05 * rng.standard_normal((len(vm0), 10))

    def loss(r):
        intr, vm = ga.apply_residuals(intr0, vm0, r)
        return ga.loss_and_grads(intr, vm, pairs, M.offsets, M.matches, w)

    L, d_intr, d_vm = loss(res)
    g = ga.residual_vjp(intr0, vm0, res, d_intr, d_vm)
    h = 1e-6
    for idx in np.ndindex(res.shape):
        r = res.copy()
        r[idx] += h
        Lp = loss(r)[0]
        r[idx] -= 2 * h
        Lm = loss(r)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * (1 + abs(fd)), (idx, fd, g[idx])
    assert np.abs(g).max() > 1e-2
