"""Seeded synthetic scenes and cameras for the rasterizer workloads.

This module only draws inputs. It holds none of the rasterizer's arithmetic,
so both the CUDA path and the FP64 oracle can be fed from it without sharing
any computation. Real datasets (MipNeRF360, Tanks-and-Temples, CO3Dv2, named
in the paper's experimental setup, Section 4.1) are not available; these
generators stand in for them with the shapes and distributions of the five
workloads:

* ``single_view_small``  : 2,000 Gaussians, SH degree 0, one 128x128 view.
* ``single_view_1m``     : 1,000,000 Gaussians in 64 clusters, SH degree 3,
                           one 1237x822 view.
* ``orbit_views``        : one 500,000-Gaussian SH3 scene seen by 16 views
                           979x546 on a circular orbit of radius 5.
* ``uneven_scenes``      : 8 scenes of 0.2M..3M Gaussians, 4 views each at
                           mixed resolutions.
* ``dense_hemisphere``   : 6M Gaussians, 300 views 1600x1066 on a hemisphere,
                           with jittered (1 degree, 1 %) initial poses.
* ``ga_cameras`` / ``ga_matches`` : cameras and keypoint correspondences for
                           the global alignment: 300 hemisphere cameras with
                           jittered initial estimates, up to 4,096 noisy
                           matches per image pair, a fraction of them outliers
                           (stand-in for a feature matcher's output).

Conventions (shared by every consumer of these arrays):

* Cameras are world->camera rigid transforms with OpenCV axes (x right,
  y down, z forward). ``viewmats[v]`` is 12 floats: the 3x3 rotation R
  row-major, then the translation t, so that x_cam = R x_world + t.
* ``intrinsics[v]`` = (fx, fy, cx, cy) in pixels.
* Quaternions are (w, x, y, z), stored unnormalised as drawn.
* SH coefficients are ``[N, (d+1)^2, 3]`` with the coefficient index
  l*l + l + m (m = -l..l) and the colour channel last.
* Views of one scene are contiguous; ``gauss_begin/gauss_count`` give the
  Gaussian range (into the concatenated arrays) that each view sees.

All sampling is numpy ``default_rng(seed)`` in float64, stored float32.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Value of the degree-0 real spherical harmonic, 1 / (2 sqrt(pi)). It only
# maps a base colour c in [0,1] to a DC coefficient (c - 0.5) / Y00, which is
# how "DC uniform" colours are drawn.
_Y00 = 0.28209479177387814


@dataclasses.dataclass
class Scene:
    means: np.ndarray           # [N,3] float32
    log_scales: np.ndarray      # [N,3] float32
    quats: np.ndarray           # [N,4] float32 (w,x,y,z), unnormalised
    opacity_logits: np.ndarray  # [N]   float32
    sh: np.ndarray              # [N,(d+1)^2,3] float32
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx], self.log_scales[idx], self.quats[idx],
                     self.opacity_logits[idx], self.sh[idx], self.sh_degree)

    def permuted(self, perm) -> "Scene":
        return self.subset(np.asarray(perm))


@dataclasses.dataclass
class Views:
    viewmats: np.ndarray     # [V,12] float32: R (row-major) then t, world->camera
    intrinsics: np.ndarray   # [V,4] float32: fx, fy, cx, cy
    width: np.ndarray        # [V] int32
    height: np.ndarray       # [V] int32
    gauss_begin: np.ndarray  # [V] int64
    gauss_count: np.ndarray  # [V] int64

    @property
    def n(self) -> int:
        return int(self.viewmats.shape[0])

    @property
    def pixels(self) -> int:
        return int(np.sum(self.width.astype(np.int64) * self.height.astype(np.int64)))

    def select(self, idx) -> "Views":
        idx = np.atleast_1d(np.asarray(idx))
        return Views(self.viewmats[idx].copy(), self.intrinsics[idx].copy(),
                     self.width[idx].copy(), self.height[idx].copy(),
                     self.gauss_begin[idx].copy(), self.gauss_count[idx].copy())


def concat_scenes(scenes) -> tuple[Scene, np.ndarray]:
    """Concatenate scenes of one SH degree; returns the scene and offsets [S+1]."""
    deg = scenes[0].sh_degree
    assert all(s.sh_degree == deg for s in scenes)
    offs = np.zeros(len(scenes) + 1, np.int64)
    offs[1:] = np.cumsum([s.n for s in scenes])
    cat = Scene(np.concatenate([s.means for s in scenes]),
                np.concatenate([s.log_scales for s in scenes]),
                np.concatenate([s.quats for s in scenes]),
                np.concatenate([s.opacity_logits for s in scenes]),
                np.concatenate([s.sh for s in scenes]), deg)
    return cat, offs


# ----------------------------------------------------------------------------
# camera helpers (pure geometry of the camera placement, not of the method)
# ----------------------------------------------------------------------------

def look_at(position, target=(0.0, 0.0, 0.0), down=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->camera [12] (R row-major, t) for an OpenCV camera at ``position``
    looking at ``target``; ``down`` is the world direction that should appear
    as image +y."""
    c = np.asarray(position, np.float64)
    f = np.asarray(target, np.float64) - c
    f /= np.linalg.norm(f)
    x = np.cross(np.asarray(down, np.float64), f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])          # rows: camera axes in world coordinates
    t = -R @ c
    return np.concatenate([R.reshape(-1), t])


def _views(viewmats, fx, width, height, begin, count) -> Views:
    viewmats = np.asarray(viewmats, np.float64).reshape(-1, 12)
    V = viewmats.shape[0]
    width = np.broadcast_to(np.asarray(width, np.int32), (V,)).copy()
    height = np.broadcast_to(np.asarray(height, np.int32), (V,)).copy()
    fx = np.broadcast_to(np.asarray(fx, np.float64), (V,))
    intr = np.stack([fx, fx, width / 2.0, height / 2.0], axis=1)
    return Views(viewmats.astype(np.float32), intr.astype(np.float32), width, height,
                 np.broadcast_to(np.asarray(begin, np.int64), (V,)).copy(),
                 np.broadcast_to(np.asarray(count, np.int64), (V,)).copy())


# ----------------------------------------------------------------------------
# Gaussian samplers
# ----------------------------------------------------------------------------

def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sh(rng, n, degree, higher_sigma):
    K = (degree + 1) ** 2
    base = rng.uniform(0.0, 1.0, (n, 3))
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = (base - 0.5) / _Y00
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, higher_sigma, (n, K - 1, 3))
    return sh


def uniform_box_scene(seed=0, n=2000, lo=(-1.0, -1.0, 2.0), hi=(1.0, 1.0, 4.0),
                      log_scale_mu=-3.0, log_scale_sigma=0.5, logit_sigma=1.0,
                      sh_degree=0, sh_sigma=0.1) -> Scene:
    rng = np.random.default_rng(seed)
    means = rng.uniform(np.asarray(lo), np.asarray(hi), (n, 3))
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, logit_sigma, n)
    sh = _sh(rng, n, sh_degree, sh_sigma)
    return Scene(means.astype(np.float32), log_scales.astype(np.float32),
                 quats.astype(np.float32), logits.astype(np.float32),
                 sh.astype(np.float32), sh_degree)


def cluster_scene(seed=0, n=1_000_000, n_clusters=64, radius=5.0, cluster_sigma=0.3,
                  log_scale_mu=-4.0, log_scale_sigma=0.7, logit_sigma=1.5,
                  sh_degree=3, sh_sigma=0.1) -> Scene:
    """Gaussian mixture of ``n_clusters`` equal-weight isotropic clusters whose
    centres are uniform in the ball of ``radius`` around the origin."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n_clusters, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.uniform(0.0, 1.0, n_clusters) ** (1.0 / 3.0)
    centres = d * r[:, None]
    which = rng.integers(0, n_clusters, n)
    means = centres[which] + rng.normal(0.0, cluster_sigma, (n, 3))
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, logit_sigma, n)
    sh = _sh(rng, n, sh_degree, sh_sigma)
    return Scene(means.astype(np.float32), log_scales.astype(np.float32),
                 quats.astype(np.float32), logits.astype(np.float32),
                 sh.astype(np.float32), sh_degree)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

def single_view_small(seed=0, n=2000):
    """2,000 Gaussians, SH0, one 128x128 view, fx=fy=150, c=64, camera at the
    origin looking +z."""
    scene = uniform_box_scene(seed, n)
    eye = np.concatenate([np.eye(3).reshape(-1), np.zeros(3)])
    views = _views(eye, 150.0, 128, 128, 0, n)
    return scene, views


def single_view_1m(seed=0, n=1_000_000, width=1237, height=822, focal=1000.0, radius=5.0):
    """1M clustered SH3 Gaussians in a ball of radius 5 (diameter 10) around the
    origin; one camera 6 units out at (0,0,-6) looking at the origin."""
    scene = cluster_scene(seed, n, radius=radius)
    views = _views(look_at((0.0, 0.0, -6.0)), focal, width, height, 0, n)
    return scene, views


def orbit_viewmats(n_views=16, radius=5.0, phase=0.0):
    out = []
    for k in range(n_views):
        th = phase + 2.0 * math.pi * k / n_views
        out.append(look_at((radius * math.sin(th), 0.0, -radius * math.cos(th))))
    return np.stack(out)


def orbit_views(seed=0, n=500_000, n_views=16, width=979, height=546, focal=1000.0):
    """One clustered SH3 scene shared by ``n_views`` cameras on the circle of
    radius 5 in the plane y=0, all looking at the origin."""
    scene = cluster_scene(seed, n)
    views = _views(orbit_viewmats(n_views), focal, width, height, 0, n)
    return scene, views


UNEVEN_SIZES = (200_000, 400_000, 800_000, 1_200_000, 1_600_000, 2_000_000, 2_500_000, 3_000_000)
UNEVEN_RESOLUTIONS = ((640, 480), (979, 546), (1237, 822), (1600, 1066))


def uneven_scenes(seeds=tuple(range(1, 9)), sizes=UNEVEN_SIZES, views_per_scene=4,
                  resolutions=UNEVEN_RESOLUTIONS, focal=1000.0):
    """Independent clustered SH3 scenes (one seed each), each seen by
    ``views_per_scene`` cameras at orbit angles 0, 90, 180, 270 degrees, with
    resolutions drawn per view from ``resolutions``."""
    scenes, vm, W, H, beg, cnt = [], [], [], [], [], []
    offs = 0
    for seed, n in zip(seeds, sizes):
        sc = cluster_scene(seed, n)
        scenes.append(sc)
        rng = np.random.default_rng(seed)
        picks = rng.choice(len(resolutions), views_per_scene)
        mats = orbit_viewmats(views_per_scene)
        for k in range(views_per_scene):
            vm.append(mats[k])
            W.append(resolutions[picks[k]][0])
            H.append(resolutions[picks[k]][1])
            beg.append(offs)
            cnt.append(n)
        offs += n
    scene, _ = concat_scenes(scenes)
    views = _views(np.stack(vm), focal, np.asarray(W), np.asarray(H),
                   np.asarray(beg), np.asarray(cnt))
    return scene, views


def hemisphere_viewmats(n_views=300, radius=5.0):
    """Fibonacci lattice on the hemisphere y <= 0 (image-up side under the
    y-down convention), every camera looking at the origin."""
    golden = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for k in range(n_views):
        y = -(k + 0.5) / n_views
        rr = math.sqrt(max(0.0, 1.0 - y * y))
        th = golden * k
        pos = radius * np.array([rr * math.cos(th), y, rr * math.sin(th)])
        out.append(look_at(pos))
    return np.stack(out)


def _axis_angle(axis, angle):
    a = np.asarray(axis, np.float64)
    a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def jitter_viewmats(viewmats, seed=0, rot_deg=1.0, trans_frac=0.01):
    """Perturb each pose by a rotation of exactly ``rot_deg`` about a uniform
    random axis (applied on the left) and a translation of ``trans_frac``*|t|
    in a uniform random direction."""
    rng = np.random.default_rng(seed)
    out = np.array(viewmats, np.float64).reshape(-1, 12).copy()
    for v in range(out.shape[0]):
        axis = rng.standard_normal(3)
        dirn = rng.standard_normal(3)
        dirn /= np.linalg.norm(dirn)
        R = out[v, :9].reshape(3, 3)
        t = out[v, 9:]
        out[v, :9] = (_axis_angle(axis, math.radians(rot_deg)) @ R).reshape(-1)
        out[v, 9:] = t + trans_frac * np.linalg.norm(t) * dirn
    return out


def dense_hemisphere(seed=0, n=6_000_000, n_views=300, width=1600, height=1066, focal=1000.0):
    """6M clustered SH3 Gaussians, 300 hemisphere cameras. Returns
    (scene, true_views, jittered_views)."""
    scene = cluster_scene(seed, n)
    mats = hemisphere_viewmats(n_views)
    true_views = _views(mats, focal, width, height, 0, n)
    noisy_views = _views(jitter_viewmats(mats, seed), focal, width, height, 0, n)
    return scene, true_views, noisy_views


def minibatch(step: int, n_views: int, batch: int = 8) -> np.ndarray:
    """View ids of training step ``step``: ``batch`` distinct views, drawn with
    ``default_rng(step)``."""
    return np.random.default_rng(step).choice(n_views, batch, replace=False)


@dataclasses.dataclass
class Matches:
    """Correspondences of a list of image pairs: the matches of pair m are
    rows ``offsets[m]:offsets[m+1]`` of ``matches`` = (x, y, x', y'), x in the
    pair's first image and x' in its second, in pixels."""
    offsets: np.ndarray   # int64 [M+1]
    matches: np.ndarray   # float32 [K,4]
    inlier: np.ndarray    # bool [K]


def ga_cameras(seed=0, n_views=300, width=1600, height=1066, focal=1000.0, rot_deg=1.0, trans_frac=0.01,
               focal_frac=0.02):
    """True cameras on the radius-5 hemisphere and initial estimates of them
    (the role of a feed-forward model's prediction): every pose jittered by
    exactly ``rot_deg`` and ``trans_frac``*|t|, every focal length scaled by
    1 + U(-focal_frac, focal_frac). Returns (true_viewmats, true_intrinsics,
    init_viewmats, init_intrinsics), all float32."""
    mats = hemisphere_viewmats(n_views)
    intr = np.tile(np.array([focal, focal, width / 2.0, height / 2.0]), (n_views, 1))
    init_mats = jitter_viewmats(mats, seed, rot_deg, trans_frac)
    rng = np.random.default_rng(seed + 1)
    init_intr = intr.copy()
    init_intr[:, :2] *= (1.0 + rng.uniform(-focal_frac, focal_frac, (n_views, 1)))
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    return f32(mats.reshape(-1, 12)), f32(intr), f32(init_mats), f32(init_intr)


def ga_points(seed=0, n=20_000, radius=2.0):
    """Scene points uniform in the ball of the given radius at the origin."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * radius * rng.uniform(0.0, 1.0, (n, 1)) ** (1.0 / 3.0)


def ga_matches(seed, points, intrinsics, viewmats, pairs, width, height, max_matches=4096, noise_px=0.5,
               outlier_frac=0.15) -> Matches:
    """For each pair (i, j): up to ``max_matches`` points visible in both TRUE
    cameras (in front, inside the image), observed with N(0, noise_px^2)
    pixel noise in both images; a fraction ``outlier_frac`` of them has x'
    replaced by a uniform position in image j."""
    rng = np.random.default_rng(seed)
    vm = np.asarray(viewmats, np.float64).reshape(-1, 12)
    K = np.asarray(intrinsics, np.float64).reshape(-1, 4)
    P = np.asarray(points, np.float64)
    uv, vis = [], []
    for n in range(vm.shape[0]):
        Xc = P @ vm[n, :9].reshape(3, 3).T + vm[n, 9:]
        z = Xc[:, 2]
        zs = np.where(z > 0.1, z, 1.0)
        u = K[n, 0] * Xc[:, 0] / zs + K[n, 2]
        v = K[n, 1] * Xc[:, 1] / zs + K[n, 3]
        uv.append(np.stack([u, v], 1))
        vis.append((z > 0.1) & (u >= 0) & (u < width) & (v >= 0) & (v < height))
    offsets = [0]
    chunks, inl = [], []
    for i, j in np.asarray(pairs).reshape(-1, 2):
        both = np.nonzero(vis[i] & vis[j])[0]
        k = min(max_matches, len(both))
        sel = rng.choice(both, k, replace=False) if k else both[:0]
        m = np.concatenate([uv[i][sel], uv[j][sel]], 1) + rng.normal(0.0, noise_px, (k, 4))
        out = rng.random(k) < outlier_frac
        m[out, 2] = rng.uniform(0, width, int(out.sum()))
        m[out, 3] = rng.uniform(0, height, int(out.sum()))
        chunks.append(m)
        inl.append(~out)
        offsets.append(offsets[-1] + k)
    matches = np.concatenate(chunks, 0) if chunks else np.zeros((0, 4))
    inlier = np.concatenate(inl) if inl else np.zeros(0, bool)
    return Matches(np.asarray(offsets, np.int64), np.ascontiguousarray(matches, np.float32), inlier)
