"""FP64 oracle of the camera global alignment (Section 3.3, Eqs. 2-4).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline); shares no code
with the CUDA library.

Cameras n = 0..N-1 have intrinsics (fx, fy, cx, cy) and world-to-camera
extrinsics (R_n, t_n), X_cam = R_n X + t_n. The steps, in the paper's order:

* candidate pairs (Sec. 3.3): pairs (i, j), i < j, whose viewing directions
  (the camera z-axis in world coordinates, the third row of R) are less than
  the angle threshold (30 degrees in Sec. 4.1) apart;
* fundamental matrix of pair m = (i, j) from the paired cameras (Eq. 2):
  R_ij = R_j R_i^T, t_ij = t_j - R_ij t_i, E = [t_ij]x R_ij,
  F_m = K_j^-T E K_i^-1, so that x'^T F_m x = 0 for a keypoint x in image i
  and its match x' in image j (homogeneous pixel coordinates (u, v, 1));
* epipolar distance (Eq. 2): e = |x'^T F x| / ||(F x)_{1,2}||, the pixel
  distance of x' to the epipolar line F x (the algebraic residual x'^T F x
  of Eq. 2 normalised so that it is a distance in pixels; a match whose
  line is undefined, (F x)_{1,2} = 0, has e = 0 and no gradient);
* loss (Eq. 2): L = sum_k w_k e_k / sum_k w_k over all pairs' matches;
* adaptive weights (Eq. 3): f is the density of a histogram of the initial
  distances with B equal bins on [0, max e]; w_k = (f(e_k) / mean_k f(e_k))^a,
  a = 0.5;
* learning rate (Eq. 4) from the median initial distance: lr0 below b1, lr2
  above b2, lr1 in between (b1, b2 inclusive in the middle band).

Decisions that turn floating point into integers (a pair passing the angle
test, a distance's histogram bin) are taken in float32, in the same
operation order the GPU uses, from the float32 inputs; everything else is
float64. Pinned in tests/test_oracle_ga.py by closed forms (zero distance for
exact matches, rank-2 F with the epipoles as null vectors), an independent
geometric construction of the distance, central differences, gauge
invariances, numpy's histogram and the median's definition.
"""
import numpy as np


def view_dirs(viewmats):
    """Camera z-axes in world coordinates: the third row of each R."""
    return np.asarray(viewmats, np.float32).reshape(-1, 12)[:, 6:9]


def select_pairs(viewmats, max_angle_deg=30.0):
    """Pairs (i, j), i < j in row-major order, with angle(d_i, d_j) below the
    threshold, i.e. d_i . d_j > cos(threshold); the dot product is evaluated
    in float32 as ((a0 b0 + a1 b1) + a2 b2), one rounding per operation."""
    d = view_dirs(viewmats)
    cos_thr = np.float32(np.cos(np.deg2rad(max_angle_deg)))
    n = d.shape[0]
    out = []
    for i in range(n):
        a = d[i]
        b = d[i + 1:]
        dot = (np.float32(a[0]) * b[:, 0] + np.float32(a[1]) * b[:, 1]).astype(np.float32)
        dot = (dot + np.float32(a[2]) * b[:, 2]).astype(np.float32)
        for j in np.nonzero(dot > cos_thr)[0]:
            out.append((i, i + 1 + int(j)))
    return np.array(out, np.int32).reshape(-1, 2)


def k_matrix(intr):
    fx, fy, cx, cy = (float(v) for v in intr)
    return np.array([[fx, 0.0, cx], [0.0, fy, cy], [0.0, 0.0, 1.0]])


def skew(t):
    return np.array([[0.0, -t[2], t[1]], [t[2], 0.0, -t[0]], [-t[1], t[0], 0.0]])


def _Rt(vm):
    vm = np.asarray(vm, np.float64)
    return vm[:9].reshape(3, 3), vm[9:12]


def relative_pose(vm_i, vm_j):
    Ri, ti = _Rt(vm_i)
    Rj, tj = _Rt(vm_j)
    R = Rj @ Ri.T
    return R, tj - R @ ti


def fundamental(intr_i, intr_j, vm_i, vm_j):
    """F = K_j^-T [t_ij]x R_ij K_i^-1 (Eq. 2)."""
    R, t = relative_pose(vm_i, vm_j)
    E = skew(t) @ R
    return np.linalg.inv(k_matrix(intr_j)).T @ E @ np.linalg.inv(k_matrix(intr_i))


def epipolar_distance(F, x, xp):
    """x, xp: [K,2] pixel coordinates in image i and j -> e [K]."""
    xh = np.concatenate([np.asarray(x, np.float64), np.ones((len(x), 1))], 1)
    xph = np.concatenate([np.asarray(xp, np.float64), np.ones((len(xp), 1))], 1)
    l = xh @ F.T
    s = np.sum(xph * l, 1)
    n = np.hypot(l[:, 0], l[:, 1])
    return np.where(n > 0, np.abs(s) / np.where(n > 0, n, 1.0), 0.0)


def distances(intr, viewmats, pairs, offsets, matches):
    """All matches' e (FP64). matches [Kt,4] = (x, y, x', y'); the matches of
    pair m are rows offsets[m]:offsets[m+1]."""
    intr = np.asarray(intr).reshape(-1, 4)
    vms = np.asarray(viewmats).reshape(-1, 12)
    out = np.zeros(len(matches))
    for m, (i, j) in enumerate(np.asarray(pairs).reshape(-1, 2)):
        a, b = int(offsets[m]), int(offsets[m + 1])
        if b > a:
            F = fundamental(intr[i], intr[j], vms[i], vms[j])
            out[a:b] = epipolar_distance(F, matches[a:b, 0:2], matches[a:b, 2:4])
    return out


def _kinv_vjp(G, intr):
    """dL/d(fx, fy, cx, cy) from dL/dK^-1 (3x3); K^-1 = [[1/fx, 0, -cx/fx],
    [0, 1/fy, -cy/fy], [0, 0, 1]]."""
    fx, fy, cx, cy = (float(v) for v in intr)
    return np.array([-G[0, 0] / fx ** 2 + G[0, 2] * cx / fx ** 2,
                     -G[1, 1] / fy ** 2 + G[1, 2] * cy / fy ** 2,
                     -G[0, 2] / fx,
                     -G[1, 2] / fy])


def loss_and_grads(intr, viewmats, pairs, offsets, matches, weights=None):
    """Eq. 2 loss and its gradient w.r.t. every camera's (fx, fy, cx, cy) and
    (R row-major, t), by the chain rule in FP64:
      de/dl = sign(s) x'/n - |s| (l1, l2, 0)/n^3    (l = F x, s = x'.l, n = |l_12|)
      dL/dF = sum_k (w_k / W) de/dl_k x_k^T
      F = B^T E A (A = K_i^-1, B = K_j^-1):  dL/dE = B G A^T,
      dL/dA = E^T B G, dL/dB = E A G^T
      E = [t]x R:  dL/dR = [t]x^T G_E,  dL/dt from M = G_E R^T as
      (M32 - M23, M13 - M31, M21 - M12)
      R = R_j R_i^T, t = t_j - R t_i:  G_R' = G_R - G_t t_i^T,
      dL/dR_j = G_R' R_i, dL/dR_i = G_R'^T R_j, dL/dt_j = G_t, dL/dt_i = -R^T G_t.
    Returns (L, d_intr [N,4], d_viewmats [N,12])."""
    intr = np.asarray(intr, np.float64).reshape(-1, 4)
    vms = np.asarray(viewmats, np.float64).reshape(-1, 12)
    matches = np.asarray(matches, np.float64)
    w = np.ones(len(matches)) if weights is None else np.asarray(weights, np.float64)
    W = w.sum()
    d_intr = np.zeros_like(intr)
    d_vm = np.zeros_like(vms)
    num = 0.0
    for m, (i, j) in enumerate(np.asarray(pairs).reshape(-1, 2)):
        a, b = int(offsets[m]), int(offsets[m + 1])
        if b <= a:
            continue
        Ai = np.linalg.inv(k_matrix(intr[i]))
        Bj = np.linalg.inv(k_matrix(intr[j]))
        R, t = relative_pose(vms[i], vms[j])
        E = skew(t) @ R
        F = Bj.T @ E @ Ai
        x = np.concatenate([matches[a:b, 0:2], np.ones((b - a, 1))], 1)
        xp = np.concatenate([matches[a:b, 2:4], np.ones((b - a, 1))], 1)
        l = x @ F.T
        s = np.sum(xp * l, 1)
        n = np.hypot(l[:, 0], l[:, 1])
        ok = n > 0
        nn = np.where(ok, n, 1.0)
        e = np.where(ok, np.abs(s) / nn, 0.0)
        num += float(np.sum(w[a:b] * e))
        g = np.where(ok, w[a:b] / W, 0.0)
        lt = np.stack([l[:, 0], l[:, 1], np.zeros(b - a)], 1)
        dedl = np.sign(s)[:, None] * xp / nn[:, None] - (np.abs(s) / nn ** 3)[:, None] * lt
        G = (g[:, None] * dedl).T @ x
        G_E = Bj @ G @ Ai.T
        G_A = E.T @ Bj @ G
        G_B = E @ Ai @ G.T
        d_intr[i] += _kinv_vjp(G_A, intr[i])
        d_intr[j] += _kinv_vjp(G_B, intr[j])
        G_R = skew(t).T @ G_E
        M = G_E @ R.T
        G_t = np.array([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]])
        Ri, ti = _Rt(vms[i])
        Rj, _ = _Rt(vms[j])
        G_R2 = G_R - np.outer(G_t, ti)
        d_vm[j, :9] += (G_R2 @ Ri).reshape(-1)
        d_vm[i, :9] += (G_R2.T @ Rj).reshape(-1)
        d_vm[j, 9:] += G_t
        d_vm[i, 9:] += -R.T @ G_t
    return num / W, d_intr, d_vm


def histogram_bins(e32, n_bins):
    """Bin of each float32 distance on [0, max e] with n_bins equal bins:
    b = min(B - 1, floor(e * (B / max e))), the quotient and the product
    each rounded to float32. All distances go to bin 0 if max e is 0."""
    e32 = np.asarray(e32, np.float32)
    emax = np.float32(e32.max()) if e32.size else np.float32(0)
    if emax <= 0:
        return np.zeros(e32.shape, np.int64), emax
    inv = np.float32(np.float32(n_bins) / emax)
    prod = (e32 * inv).astype(np.float32)
    return np.minimum(n_bins - 1, np.floor(prod).astype(np.int64)), emax


def pdf_weights(e32, n_bins=100, alpha=0.5):
    """Eq. 3: w_k = (f(e_k) / mean_k f(e_k))^alpha with f the histogram
    density (count / (K * bin width)). Returns (w [K], counts [B])."""
    K = len(e32)
    idx, emax = histogram_bins(e32, n_bins)
    counts = np.bincount(idx, minlength=n_bins)[:n_bins] if K else np.zeros(n_bins, np.int64)
    if K == 0:
        return np.zeros(0), counts
    width = float(emax) / n_bins if emax > 0 else 1.0
    dens = counts / (K * width)
    f = dens[idx]
    return (f / f.mean()) ** alpha, counts


def median_order_stats(e32):
    """The two middle order statistics (equal for an odd count) and the
    median, their mean, in FP64."""
    s = np.sort(np.asarray(e32, np.float32))
    K = len(s)
    lo, hi = s[(K - 1) // 2], s[K // 2]
    return float(lo), float(hi), 0.5 * (float(lo) + float(hi))


def lr_rule(median, lr=(5e-4, 1e-3, 1e-2), b=(2.5, 7.5)):
    """Eq. 4 with the Sec. 4.1 constants."""
    if median < b[0]:
        return lr[0]
    if median > b[1]:
        return lr[2]
    return lr[1]


def rotation_6d(a):
    """6D rotation residual (Section 3.4) -> 3x3: b1 = a1/|a1|,
    b2 = normalise(a2 - (b1.a2) b1), b3 = b1 x b2, as columns."""
    a = np.asarray(a, np.float64)
    b1 = a[:3] / np.linalg.norm(a[:3])
    u = a[3:] - (b1 @ a[3:]) * b1
    b2 = u / np.linalg.norm(u)
    return np.stack([b1, b2, np.cross(b1, b2)], 1)


def apply_residuals(intr0, vm0, res, optimise_focal=True):
    """Cameras from per-camera residuals res [N,10] = (6D rotation,
    translation, log focal): R' = dR R, t' = t + dt, (fx', fy') =
    (fx, fy) exp(df) (df ignored unless optimise_focal)."""
    intr0 = np.asarray(intr0, np.float64).reshape(-1, 4)
    vm0 = np.asarray(vm0, np.float64).reshape(-1, 12)
    res = np.asarray(res, np.float64).reshape(-1, 10)
    intr = intr0.copy()
    vm = vm0.copy()
    for n in range(len(vm0)):
        vm[n, :9] = (rotation_6d(res[n, :6]) @ vm0[n, :9].reshape(3, 3)).reshape(-1)
        vm[n, 9:] = vm0[n, 9:] + res[n, 6:9]
        if optimise_focal:
            intr[n, :2] = intr0[n, :2] * np.exp(res[n, 9])
    return intr, vm


def residual_vjp(intr0, vm0, res, d_intr, d_vm, optimise_focal=True):
    """dL/d(residuals) [N,10] from dL/d(intrinsics) and dL/d(viewmats) at
    apply_residuals(...), by the chain rule through the Gram-Schmidt map:
      G_dR = G_R' R^T (columns g1, g2, g3), b3 = b1 x b2:
        g1 += b2 x g3, g2 += g3 x b1;
      b2 = u/|u|: g_u = (g2 - b2 (b2.g2))/|u|;
      u = a2 - (b1.a2) b1: g_a2 = g_u - (b1.g_u) b1, g1 += -(b1.a2) g_u - (b1.g_u) a2;
      b1 = a1/|a1|: g_a1 = (g1 - b1 (b1.g1))/|a1|;
      dt: G_t'; df: fx' dL/dfx' + fy' dL/dfy'."""
    intr0 = np.asarray(intr0, np.float64).reshape(-1, 4)
    vm0 = np.asarray(vm0, np.float64).reshape(-1, 12)
    res = np.asarray(res, np.float64).reshape(-1, 10)
    d_intr = np.asarray(d_intr, np.float64).reshape(-1, 4)
    d_vm = np.asarray(d_vm, np.float64).reshape(-1, 12)
    out = np.zeros_like(res)
    for n in range(len(res)):
        a1, a2 = res[n, :3], res[n, 3:6]
        n1 = np.linalg.norm(a1)
        b1 = a1 / n1
        s = b1 @ a2
        u = a2 - s * b1
        nu = np.linalg.norm(u)
        b2 = u / nu
        G = d_vm[n, :9].reshape(3, 3) @ vm0[n, :9].reshape(3, 3).T
        g1, g2, g3 = G[:, 0].copy(), G[:, 1].copy(), G[:, 2].copy()
        g1 += np.cross(b2, g3)
        g2 += np.cross(g3, b1)
        gu = (g2 - b2 * (b2 @ g2)) / nu
        ga2 = gu - (b1 @ gu) * b1
        g1 += -s * gu - (b1 @ gu) * a2
        out[n, :3] = (g1 - b1 * (b1 @ g1)) / n1
        out[n, 3:6] = ga2
        out[n, 6:9] = d_vm[n, 9:]
        if optimise_focal:
            f = intr0[n, :2] * np.exp(res[n, 9])
            out[n, 9] = d_intr[n, 0] * f[0] + d_intr[n, 1] * f[1]
    return out
