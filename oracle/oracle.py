"""Python face of the FP64 oracle (``gs_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg; never by the product package. It shares no
code with the CUDA library. Inputs are upcast to float64 here, the C code
computes everything in float64 except the binning, which is specified in
float32 (tile rectangles and sort keys) and emulated exactly.

Paper anchors: Section 3.1 (Gaussian primitive, alpha blending), Section 3.4
(per-view pose residuals whose gradients the backward provides).

Functions and what pins them (the tests under ``tests/``):

* ``sh_basis``        -- pinned against ``scipy.special.sph_harm_y`` and
                         quadrature orthonormality.
* ``project_view``    -- pinned by the on-axis isotropic closed form, Monte
                         Carlo moments of projected samples, eigen-structure
                         of Sigma, finite differences.
* ``bin_view``        -- pinned by brute-force tile/square overlap tests.
* ``render_view``     -- pinned by single-Gaussian peak, stacked
                         transmittance, early stop, alpha cutoff/clamp,
                         numpy brute-force compositing, permutation,
                         tile-size and translation invariance.
* ``render_bwd_view`` / ``project_bwd_view`` / ``pose_twist`` -- pinned by
                         FP64 central finite differences and by an
                         independent torch autograd restatement.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FLAG_GATE, FLAG_ALPHA, FLAG_T, FLAG_DEPTH, FLAG_CLAMP, FLAG_RADIUS = 1, 2, 4, 8, 16, 32
# flags that make a pixel's FP32 image legitimately differ from FP64
IMAGE_FLAGS = FLAG_GATE | FLAG_ALPHA | FLAG_T | FLAG_DEPTH | FLAG_RADIUS
# flags that make its gradient differ (adds the opacity-clamp switch)
GRAD_FLAGS = IMAGE_FLAGS | FLAG_CLAMP


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C11, no FMA contraction so that the
    float32 binning emulation rounds exactly once per operation)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Params(ctypes.Structure):
    _fields_ = [("near_z", ctypes.c_double), ("dilation", ctypes.c_double),
                ("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double),
                ("t_min", ctypes.c_double), ("fov_clamp", ctypes.c_double),
                ("bg", ctypes.c_double * 3), ("pixel_gate", ctypes.c_int),
                ("eps_gate", ctypes.c_double), ("eps_alpha", ctypes.c_double),
                ("eps_t", ctypes.c_double), ("eps_depth", ctypes.c_double),
                ("eps_clamp", ctypes.c_double)]


class _Cam(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("W", ctypes.c_int), ("H", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.or_bin_count.restype = ctypes.c_int64
    return _lib


@dataclasses.dataclass
class Params:
    near: float = 0.2
    dilation: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    fov_clamp: float = 1.3
    bg: tuple = (0.0, 0.0, 0.0)
    pixel_gate: bool = True
    # Margins that flag pixels where an FP32 evaluation may take the other
    # side of a threshold. FP32 rounding is 2^-24 ~ 6e-8 relative per
    # operation; ~100 sequential transmittance products accumulate ~1e-5,
    # hence 5e-5 relative for the alpha/T decisions. The gate margin covers
    # the ~1e-5 px error of a compensated float32 mean.
    eps_gate: float = 1e-4
    eps_alpha: float = 5e-5
    eps_t: float = 5e-5
    eps_depth: float = 1e-6
    eps_clamp: float = 5e-5

    def c(self) -> _Params:
        return _Params(self.near, self.dilation, self.alpha_min, self.alpha_max, self.t_min,
                       self.fov_clamp, (ctypes.c_double * 3)(*self.bg), int(self.pixel_gate),
                       self.eps_gate, self.eps_alpha, self.eps_t, self.eps_depth, self.eps_clamp)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def camera(viewmat, intr, W, H) -> _Cam:
    vm = np.asarray(viewmat, np.float64)
    it = np.asarray(intr, np.float64)
    return _Cam((ctypes.c_double * 9)(*vm[:9]), (ctypes.c_double * 3)(*vm[9:12]),
                float(it[0]), float(it[1]), float(it[2]), float(it[3]), int(W), int(H))


def view_camera(views, v) -> _Cam:
    return camera(views.viewmats[v], views.intrinsics[v], views.width[v], views.height[v])


def sh_basis(degree: int, d):
    d = _f64(d)
    Y = np.zeros(16)
    dY = np.zeros(48)
    lib().or_sh_basis(ctypes.c_int(degree), _p(d), _p(Y), _p(dY))
    K = (degree + 1) ** 2
    return Y[:K], dY.reshape(16, 3)[:K]


def _scene_arrays(scene, begin=0, count=None):
    count = scene.n - begin if count is None else count
    sl = slice(begin, begin + count)
    return (_f64(scene.means[sl]), _f64(scene.log_scales[sl]), _f64(scene.quats[sl]),
            _f64(scene.opacity_logits[sl]), _f64(scene.sh[sl]))


def project_view(scene, views, v, params: Params = None, threads: int = 1):
    """Projection of the Gaussians view ``v`` sees (local indices); with
    threads > 1 the same work split over that many threads (for timing)."""
    params = params or Params()
    b, c = int(views.gauss_begin[v]), int(views.gauss_count[v])
    means, ls, q, lg, sh = _scene_arrays(scene, b, c)
    n = c
    out = dict(xy=np.zeros((n, 2)), depth=np.zeros(n), conic=np.zeros((n, 3)), cov=np.zeros((n, 3)),
               opac=np.zeros(n), rgb=np.zeros((n, 3)), radius=np.zeros(n, np.int32),
               r_real=np.zeros(n), clamped=np.zeros((n, 3), np.int32), ext=np.zeros((n, 2)))
    cam = view_camera(views, v)
    prm = params.c()
    args = (ctypes.c_int64(n), ctypes.c_int(scene.sh_degree), _p(means), _p(ls), _p(q), _p(lg),
            _p(sh), ctypes.byref(cam), ctypes.byref(prm),
            _p(out["xy"]), _p(out["depth"]), _p(out["conic"]), _p(out["cov"]), _p(out["opac"]),
            _p(out["rgb"]), _p(out["radius"]), _p(out["r_real"]), _p(out["clamped"]), _p(out["ext"]))
    if threads > 1:
        lib().or_project_mt(*args, ctypes.c_int(threads))
    else:
        lib().or_project(*args)
    return out


def tile_grid(W, H, TW, TH):
    return (W + TW - 1) // TW, (H + TH - 1) // TH


def bin_view(x, y, r, depth, W, H, TW=16, TH=16, ext=None):
    """Float32 binning: ranges [G,2] (tile id ty*Gx+tx), keys uint64
    (depth bits << 32 | local index) ascending per tile, ids int32. The tile
    rectangle's half-extents are ext [n,2] (float32), or r if ext is None."""
    x = np.ascontiguousarray(x, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    depth = np.ascontiguousarray(depth, np.float32)
    r = np.ascontiguousarray(r, np.int32)
    if ext is None:
        ext = np.stack([r, r], axis=1)
    ext = np.ascontiguousarray(ext, np.float32)
    n = x.shape[0]
    Gx, Gy = tile_grid(W, H, TW, TH)
    counts = np.zeros(Gx * Gy, np.int32)
    total = lib().or_bin_count(ctypes.c_int64(n), _p(x), _p(y), _p(r), _p(ext), W, H, TW, TH, _p(counts))
    ranges = np.zeros((Gx * Gy, 2), np.int64)
    keys = np.zeros(max(total, 1), np.uint64)
    ids = np.zeros(max(total, 1), np.int32)
    lib().or_bin_fill(ctypes.c_int64(n), _p(x), _p(y), _p(r), _p(ext), _p(depth), W, H, TW, TH,
                      _p(ranges), _p(keys), _p(ids))
    return ranges, keys[:total], ids[:total]


def bins_for_render(proj, W, H, TW, TH, params: Params = None):
    """Tile lists for rendering: float32-rounded means/depths and extents
    enlarged by a hair (and by one pixel where 3 sqrt(lambda) sits within the
    gate margin of an integer), so that every Gaussian a float32 evaluation
    could list is present. The lists only bound the search: compositing
    applies the radius gate and the alpha rule itself."""
    params = params or Params()
    r = proj["radius"].copy()
    fr = proj["r_real"] - np.floor(proj["r_real"])
    amb = (r > 0) & ((fr < params.eps_gate) | (fr > 1 - params.eps_gate))
    ext = proj["ext"] * (1 + 1e-5) + 1e-4
    ext[amb] += 1.0
    return bin_view(proj["xy"][:, 0], proj["xy"][:, 1], r, proj["depth"], W, H, TW, TH, ext)


def render_view(proj, W, H, TW=16, TH=16, params: Params = None, bins=None, mask=None, threads: int = 1):
    """mask: optional [H,W] bool; only those pixels are computed (others 0).
    threads > 1: rows of tiles interleaved over that many threads (timing)."""
    params = params or Params()
    if bins is None:
        bins = bins_for_render(proj, W, H, TW, TH, params)
    ranges, _, ids = bins
    img = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    fl = np.zeros((H, W), np.int32)
    prm = params.c()
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    args = (_p(proj["xy"]), _p(proj["conic"]), _p(proj["opac"]), _p(proj["rgb"]),
            _p(proj["radius"]), _p(proj["r_real"]), _p(proj["depth"]), W, H, TW, TH,
            _p(np.ascontiguousarray(ranges)), _p(np.ascontiguousarray(ids)), ctypes.byref(prm),
            None if m is None else _p(m), _p(img), _p(T), _p(nc), _p(fl))
    if threads > 1:
        lib().or_render_mt(*args, ctypes.c_int(threads))
    else:
        lib().or_render(*args)
    return dict(image=img, T=T, n_contrib=nc, flags=fl)


def render_bwd_view(proj, W, H, dL_dimg, TW=16, TH=16, params: Params = None, bins=None, threads: int = 1):
    params = params or Params()
    if bins is None:
        bins = bins_for_render(proj, W, H, TW, TH, params)
    ranges, _, ids = bins
    n = proj["xy"].shape[0]
    g2d = np.zeros((n, 9))
    prm = params.c()
    args = (ctypes.c_int64(n), _p(proj["xy"]), _p(proj["conic"]), _p(proj["opac"]),
            _p(proj["rgb"]), _p(proj["radius"]), _p(proj["depth"]), W, H, TW, TH,
            _p(np.ascontiguousarray(ranges)), _p(np.ascontiguousarray(ids)), ctypes.byref(prm),
            _p(_f64(dL_dimg)), _p(g2d))
    if threads > 1:
        if lib().or_render_bwd_mt(*args, ctypes.c_int(threads)) != 0:
            raise MemoryError("or_render_bwd_mt: per-thread scratch")
    else:
        lib().or_render_bwd(*args)
    return g2d


def project_bwd_view(scene, views, v, g2d, params: Params = None, threads: int = 1):
    """Raw-parameter gradients of the Gaussians view ``v`` sees (local
    indices) and the view's dL/dR [9], dL/dt [3]."""
    params = params or Params()
    b, c = int(views.gauss_begin[v]), int(views.gauss_count[v])
    means, ls, q, lg, sh = _scene_arrays(scene, b, c)
    K = (scene.sh_degree + 1) ** 2
    out = dict(means=np.zeros((c, 3)), log_scales=np.zeros((c, 3)), quats=np.zeros((c, 4)),
               opacity_logits=np.zeros(c), sh=np.zeros((c, K, 3)))
    gR = np.zeros(9)
    gt = np.zeros(3)
    cam = view_camera(views, v)
    prm = params.c()
    args = (ctypes.c_int64(c), ctypes.c_int(scene.sh_degree), _p(means), _p(ls), _p(q), _p(lg),
            _p(sh), ctypes.byref(cam), ctypes.byref(prm), _p(_f64(g2d)),
            _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]),
            _p(out["opacity_logits"]), _p(out["sh"]), _p(gR), _p(gt))
    if threads > 1:
        lib().or_project_bwd_mt(*args, ctypes.c_int(threads))
    else:
        lib().or_project_bwd(*args)
    return out, gR, gt


def pose_twist(viewmat, gR, gt):
    vm = _f64(viewmat)
    R = np.ascontiguousarray(vm[:9])
    t = np.ascontiguousarray(vm[9:12])
    tw = np.zeros(6)
    lib().or_pose_twist(_p(R), _p(t), _p(_f64(gR)), _p(_f64(gt)), _p(tw))
    return tw


# ---------------------------------------------------------------------------
# whole-path helpers
# ---------------------------------------------------------------------------

def forward(scene, views, TW=16, TH=16, params: Params = None, masks=None, threads: int = 1):
    """Per view: projection, tile lists and rendering. Returns a list of dicts
    with keys proj, bins, image [3,H,W], T, n_contrib, flags. masks: optional
    per-view [H,W] bool arrays restricting the rendered pixels. threads > 1
    splits projection and rendering over that many threads (for timing; the
    binning stays single-threaded)."""
    params = params or Params()
    out = []
    for v in range(views.n):
        W, H = int(views.width[v]), int(views.height[v])
        proj = project_view(scene, views, v, params, threads)
        bins = bins_for_render(proj, W, H, TW, TH, params)
        r = render_view(proj, W, H, TW, TH, params, bins, None if masks is None else masks[v], threads)
        r.update(proj=proj, bins=bins)
        out.append(r)
    return out


def backward(scene, views, fwd, dL_dimgs, TW=16, TH=16, params: Params = None, threads: int = 1):
    """Gradients of sum_v <dL_dimgs[v], image_v> w.r.t. every raw parameter
    (global indexing) and every view's R, t (dL_dRt [V,12]) and twist [V,6];
    threads > 1 as in forward()."""
    params = params or Params()
    K = (scene.sh_degree + 1) ** 2
    N = scene.n
    grads = dict(means=np.zeros((N, 3)), log_scales=np.zeros((N, 3)), quats=np.zeros((N, 4)),
                 opacity_logits=np.zeros(N), sh=np.zeros((N, K, 3)))
    dRt = np.zeros((views.n, 12))
    tw = np.zeros((views.n, 6))
    g2ds = []
    for v in range(views.n):
        W, H = int(views.width[v]), int(views.height[v])
        f = fwd[v]
        g2d = render_bwd_view(f["proj"], W, H, dL_dimgs[v], TW, TH, params, f["bins"], threads)
        g2ds.append(g2d)
        gv, gR, gt = project_bwd_view(scene, views, v, g2d, params, threads)
        b, c = int(views.gauss_begin[v]), int(views.gauss_count[v])
        for k in grads:
            grads[k][b:b + c] += gv[k]
        dRt[v, :9] = gR
        dRt[v, 9:] = gt
        tw[v] = pose_twist(views.viewmats[v], gR, gt)
    return grads, dRt, tw, g2ds
