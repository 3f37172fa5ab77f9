"""ctypes binding of libgsplat_gb300.so (include/gs.h), same names as the C ABI.

Argument marshalling only: every step of the rasterizer runs in the CUDA
library. torch provides device memory and the current stream. There is no
fallback: if the library is missing or the device is not CUDA, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsplat_gb300.so")

GS_OK, GS_ERR_ARG, GS_ERR_CUDA, GS_ERR_CAPACITY, GS_ERR_UNSUPPORTED, GS_ERR_OVERFLOW, GS_ERR_TOO_LARGE, GS_ERR_TIMEOUT = range(8)
GS_MAX_VIEWS = 64
GS_RECORD_FLOATS = 16
GS_GRAD2D_FLOATS = 12
GS_NUM_COUNTERS = 16

EXPORTED = ["gs_config_default", "gs_num_slots", "gs_slot_base", "gs_num_tiles", "gs_tile_base",
            "gs_num_image_floats", "gs_pixel_base", "gs_pose_blocks", "gs_project", "gs_bin_sort",
            "gs_render_fwd", "gs_render_bwd", "gs_rasterize_bwd", "gs_rasterize_bwd_l1", "gs_project_bwd", "gs_pose_grad", "gs_l1_loss", "gs_error_string", "gs_version",
            "gs_project_bwd_noalloc", "gs_sgld_adam_step", "gs_ga_select_pairs", "gs_ga_incidence",
            "gs_ga_epipolar", "gs_ga_weights_scratch_bytes", "gs_ga_weights", "gs_ga_step", "gs_l1_dssim_loss",
            "gs_check_bounded_wait", "gs_workspace_size", "gs_workspace_carve", "gs_status_read",
            "gs_probe_blocks", "gs_peak_probe", "gs_spatial_codes"]
GS_GA_MAX_CAMS = 8192
GS_GA_PAIR_FLOATS = 12
GS_GA_MAX_BINS = 16384
GS_MAX_ADAM_GROUPS = 8


class GsError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {error_string(code)} (code {code})")
        self.code = code


class gs_config(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("pixel_gate", ctypes.c_int),
                ("near_z", ctypes.c_float), ("dilation", ctypes.c_float), ("alpha_min", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("t_min", ctypes.c_float), ("fov_clamp", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("count_pairs", ctypes.c_int), ("accumulate_grads", ctypes.c_int),
                ("use_tma", ctypes.c_int), ("fwd_batch", ctypes.c_int), ("bwd_batch", ctypes.c_int),
                ("overlap_prev", ctypes.c_int)]


class gs_gaussians(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int), ("means", ctypes.c_void_p),
                ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class gs_views(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int), ("viewmats", ctypes.c_void_p), ("intrinsics", ctypes.c_void_p),
                ("width", ctypes.c_void_p), ("height", ctypes.c_void_p), ("gauss_begin", ctypes.c_void_p),
                ("gauss_count", ctypes.c_void_p)]


class gs_bins(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("tile_ranges", ctypes.c_void_p), ("keys", ctypes.c_void_p),
                ("ids", ctypes.c_void_p), ("keys_tmp", ctypes.c_void_p), ("tile_order", ctypes.c_void_p),
                ("tile_scratch", ctypes.c_void_p), ("counters", ctypes.c_void_p), ("last_contrib", ctypes.c_void_p),
                ("tile_work", ctypes.c_void_p)]


class gs_adam_group(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("exp_avg", ctypes.c_void_p),
                ("exp_avg_sq", ctypes.c_void_p), ("count", ctypes.c_int64), ("lr", ctypes.c_float)]


class gs_ga_problem(ctypes.Structure):
    _fields_ = [("n_cams", ctypes.c_int), ("intrinsics", ctypes.c_void_p), ("viewmats", ctypes.c_void_p),
                ("n_pairs", ctypes.c_int64), ("pairs", ctypes.c_void_p), ("match_offsets", ctypes.c_void_p),
                ("n_matches", ctypes.c_int64), ("matches", ctypes.c_void_p), ("weights", ctypes.c_void_p)]


class gs_ga_state(ctypes.Structure):
    _fields_ = [("n_cams", ctypes.c_int), ("intrinsics0", ctypes.c_void_p), ("viewmats0", ctypes.c_void_p),
                ("residuals", ctypes.c_void_p), ("exp_avg", ctypes.c_void_p), ("exp_avg_sq", ctypes.c_void_p),
                ("step", ctypes.c_void_p), ("intrinsics", ctypes.c_void_p), ("viewmats", ctypes.c_void_p),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double), ("optimise_focal", ctypes.c_int)]


class gs_grads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity_logits", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("grad2d", ctypes.c_void_p),
                ("pose_partials", ctypes.c_void_p)]


_lib = None


def load():
    """Load the library (built by ``__graft_entry__.build()`` or
    ``paper_2509_25191_gb300.build``). Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgsplat_gb300.so not built ({LIB_PATH} missing); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name in ["gs_num_slots", "gs_slot_base", "gs_num_tiles", "gs_tile_base", "gs_num_image_floats",
                 "gs_pixel_base"]:
        getattr(lib, name).restype = ctypes.c_int64
    lib.gs_error_string.restype = ctypes.c_char_p
    lib.gs_ga_weights_scratch_bytes.restype = ctypes.c_size_t
    lib.gs_workspace_size.restype = ctypes.c_size_t
    lib.gs_workspace_size.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64]
    lib.gs_workspace_carve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]
    _lib = lib
    return lib


def error_string(code: int) -> str:
    try:
        return load().gs_error_string(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


def _check(rc, where):
    if rc != GS_OK:
        raise GsError(rc, where)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------------------
# argument structures
# ---------------------------------------------------------------------------

def config(tile=(16, 16), pixel_gate=True, bg=(0.0, 0.0, 0.0), near=0.2, dilation=0.3,
           alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=1e-4, fov_clamp=1.3, count_pairs=False,
           accumulate_grads=False, use_tma=True, batch=(2, 1), overlap_prev=False) -> gs_config:
    c = gs_config()
    load().gs_config_default(ctypes.byref(c))
    c.tile_w, c.tile_h = int(tile[0]), int(tile[1])
    c.pixel_gate = int(bool(pixel_gate))
    c.near_z, c.dilation, c.alpha_min, c.alpha_max, c.t_min, c.fov_clamp = \
        near, dilation, alpha_min, alpha_max, t_min, fov_clamp
    c.bg = (ctypes.c_float * 3)(*bg)
    c.count_pairs = int(bool(count_pairs))
    c.accumulate_grads = int(bool(accumulate_grads))
    c.use_tma = int(bool(use_tma))
    c.fwd_batch, c.bwd_batch = int(batch[0]), int(batch[1])
    c.overlap_prev = int(bool(overlap_prev))
    return c


class Gaussians:
    """Device tensors of the Gaussians (float32, contiguous, on one CUDA device)."""

    def __init__(self, means, log_scales, quats, opacity_logits, sh):
        self.means, self.log_scales, self.quats = means, log_scales, quats
        self.opacity_logits, self.sh = opacity_logits, sh
        K = sh.shape[1]
        self.sh_degree = int(round(K ** 0.5)) - 1
        assert (self.sh_degree + 1) ** 2 == K and sh.shape[2] == 3
        self.n = int(means.shape[0])
        for t in (means, log_scales, quats, opacity_logits, sh):
            assert t.dtype == torch.float32 and t.is_cuda and t.is_contiguous()

    def c(self) -> gs_gaussians:
        return gs_gaussians(self.n, self.sh_degree, _ptr(self.means), _ptr(self.log_scales), _ptr(self.quats),
                            _ptr(self.opacity_logits), _ptr(self.sh))

    @staticmethod
    def from_scene(scene, device="cuda"):
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device)
        return Gaussians(f(scene.means), f(scene.log_scales), f(scene.quats), f(scene.opacity_logits), f(scene.sh))


class Views:
    """Views of one call: device pose/intrinsics tensors plus host layout."""

    def __init__(self, viewmats, intrinsics, width, height, gauss_begin, gauss_count):
        self.viewmats, self.intrinsics = viewmats, intrinsics
        self.width = np.ascontiguousarray(width, np.int32)
        self.height = np.ascontiguousarray(height, np.int32)
        self.gauss_begin = np.ascontiguousarray(gauss_begin, np.int64)
        self.gauss_count = np.ascontiguousarray(gauss_count, np.int64)
        self.n = int(self.width.shape[0])
        assert 1 <= self.n <= GS_MAX_VIEWS

    def c(self) -> gs_views:
        return gs_views(self.n, _ptr(self.viewmats), _ptr(self.intrinsics),
                        self.width.ctypes.data_as(ctypes.c_void_p), self.height.ctypes.data_as(ctypes.c_void_p),
                        self.gauss_begin.ctypes.data_as(ctypes.c_void_p),
                        self.gauss_count.ctypes.data_as(ctypes.c_void_p))

    @staticmethod
    def from_synth(views, device="cuda", viewmats=None):
        vm = viewmats if viewmats is not None else torch.as_tensor(views.viewmats, dtype=torch.float32).to(device)
        return Views(vm.contiguous(), torch.as_tensor(views.intrinsics, dtype=torch.float32).to(device),
                     views.width, views.height, views.gauss_begin, views.gauss_count)

    # layout
    def num_slots(self):
        return int(self.gauss_count.sum())

    def slot_base(self, v):
        return int(self.gauss_count[:v].sum())

    def num_tiles(self, cfg):
        return int(load().gs_num_tiles(ctypes.byref(self.c()), ctypes.byref(cfg)))

    def tile_base(self, cfg, v):
        return int(load().gs_tile_base(ctypes.byref(self.c()), ctypes.byref(cfg), v))

    def num_image_floats(self):
        return int(3 * (self.width.astype(np.int64) * self.height).sum())

    def pixel_base(self, v):
        return int(3 * (self.width[:v].astype(np.int64) * self.height[:v]).sum())

    @property
    def pixels(self):
        return int((self.width.astype(np.int64) * self.height).sum())


class Bins:
    """Caller-owned tile-list buffers (device). With pixels > 0 the per-pixel
    last-contributor record is kept too (the forward writes it, the backward
    ends each pixel's replay there), and the per-tile work record (each
    forward orders its tiles by the previous forward's replay lengths and
    writes its own)."""

    def __init__(self, n_tiles, capacity, device="cuda", pixels=0):
        self.n_tiles, self.capacity, self.pixels = int(n_tiles), int(capacity), int(pixels)
        i32 = dict(dtype=torch.int32, device=device)
        self.tile_ranges = torch.empty(max(1, self.n_tiles) * 2, **i32)
        self.tile_order = torch.empty(max(1, self.n_tiles), **i32)
        self.tile_scratch = torch.empty(max(1, 5 * self.n_tiles), **i32)
        self.counters = torch.zeros(GS_NUM_COUNTERS, **i32)
        cap = max(1, self.capacity)
        self.keys = torch.empty(cap, dtype=torch.int64, device=device)
        self.keys_tmp = torch.empty(cap, dtype=torch.int64, device=device)
        self.ids = torch.empty(cap, dtype=torch.int32, device=device)
        self.last_contrib = torch.empty(self.pixels, **i32) if self.pixels > 0 else None
        self.tile_work = torch.zeros(max(1, self.n_tiles), **i32) if self.pixels > 0 else None

    def c(self, last=True) -> gs_bins:
        """The C struct; last=False leaves the last-contributor record out
        (NULL), e.g. for a backward whose forward wrote another image."""
        return gs_bins(self.capacity, _ptr(self.tile_ranges), _ptr(self.keys), _ptr(self.ids), _ptr(self.keys_tmp),
                       _ptr(self.tile_order), _ptr(self.tile_scratch), _ptr(self.counters),
                       _ptr(self.last_contrib) if last else None, _ptr(self.tile_work) if last else None)


class Grads:
    """Gradient outputs and backward scratch (device)."""

    def __init__(self, n, sh_degree, n_slots, n_views, device="cuda", want_gaussian_grads=True):
        K = (sh_degree + 1) ** 2
        f = dict(dtype=torch.float32, device=device)
        nn = max(1, n) if want_gaussian_grads else 1
        self.means = torch.empty(nn, 3, **f)
        self.log_scales = torch.empty(nn, 3, **f)
        self.quats = torch.empty(nn, 4, **f)
        self.opacity_logits = torch.empty(nn, **f)
        self.sh = torch.empty(nn, K, 3, **f)
        self.grad2d = torch.empty(max(1, n_slots), GS_GRAD2D_FLOATS, **f)
        self.n_blocks = int(load().gs_pose_blocks(ctypes.c_int64(n)))
        self.pose_partials = torch.empty(n_views * self.n_blocks * 12, **f)

    def c(self) -> gs_grads:
        return gs_grads(_ptr(self.means), _ptr(self.log_scales), _ptr(self.quats), _ptr(self.opacity_logits),
                        _ptr(self.sh), _ptr(self.grad2d), _ptr(self.pose_partials))


def new_status(device="cuda"):
    return torch.zeros(4, dtype=torch.int32, device=device)


# ---------------------------------------------------------------------------
# the C ABI, one wrapper per entry point
# ---------------------------------------------------------------------------

def gs_project(g: Gaussians, views: Views, cfg: gs_config, proj, status=None, stream=None):
    _check(load().gs_project(ctypes.byref(g.c()), ctypes.byref(views.c()), ctypes.byref(cfg), _ptr(proj),
                             _ptr(status), _stream(stream)), "gs_project")


def gs_bin_sort(views: Views, cfg: gs_config, proj, bins: Bins, status=None, stream=None):
    _check(load().gs_bin_sort(ctypes.byref(views.c()), ctypes.byref(cfg), _ptr(proj), ctypes.byref(bins.c()),
                              _ptr(status), _stream(stream)), "gs_bin_sort")


def gs_render_fwd(views: Views, cfg: gs_config, proj, bins: Bins, image, status=None, stream=None):
    _check(load().gs_render_fwd(ctypes.byref(views.c()), ctypes.byref(cfg), _ptr(proj), ctypes.byref(bins.c()),
                                _ptr(image), _ptr(status), _stream(stream)), "gs_render_fwd")


def gs_render_bwd(g: Gaussians, views: Views, cfg: gs_config, proj, bins: Bins, image, dL_dimage, grads: Grads,
                  want_gaussian_grads=True, status=None, stream=None, use_last=True):
    _check(load().gs_render_bwd(ctypes.byref(g.c()), ctypes.byref(views.c()), ctypes.byref(cfg), _ptr(proj),
                                ctypes.byref(bins.c(use_last)), _ptr(image), _ptr(dL_dimage),
                                ctypes.byref(grads.c()), int(bool(want_gaussian_grads)), _ptr(status),
                                _stream(stream)), "gs_render_bwd")


def gs_rasterize_bwd(views: Views, cfg: gs_config, proj, bins: Bins, image, dL_dimage, grad2d, status=None,
                     stream=None, use_last=True):
    _check(load().gs_rasterize_bwd(ctypes.byref(views.c()), ctypes.byref(cfg), _ptr(proj),
                                   ctypes.byref(bins.c(use_last)), _ptr(image), _ptr(dL_dimage), _ptr(grad2d),
                                   _ptr(status), _stream(stream)), "gs_rasterize_bwd")


def gs_rasterize_bwd_l1(views: Views, cfg: gs_config, proj, bins: Bins, image, target, loss, grad2d, status=None,
                        stream=None, use_last=True):
    """The raster backward of the mean L1 loss against target, the loss
    folded in (loss[0] = mean |image - target|; no dL/dimage buffer)."""
    _check(load().gs_rasterize_bwd_l1(ctypes.byref(views.c()), ctypes.byref(cfg), _ptr(proj),
                                      ctypes.byref(bins.c(use_last)), _ptr(image), _ptr(target), _ptr(loss),
                                      _ptr(grad2d), _ptr(status), _stream(stream)), "gs_rasterize_bwd_l1")


def gs_project_bwd(g: Gaussians, views: Views, cfg: gs_config, proj, grads: Grads, want_gaussian_grads=True,
                   status=None, stream=None):
    _check(load().gs_project_bwd(ctypes.byref(g.c()), ctypes.byref(views.c()), ctypes.byref(cfg), _ptr(proj),
                                 _ptr(grads.grad2d), ctypes.byref(grads.c()), int(bool(want_gaussian_grads)),
                                 _ptr(status), _stream(stream)), "gs_project_bwd")


def gs_project_bwd_noalloc(g: Gaussians, views: Views, cfg: gs_config, proj, grads: Grads, dL_dviewmat,
                           dL_dtwist=None, want_gaussian_grads=True, status=None, stream=None):
    """gs_project_bwd + gs_pose_grad without caller scratch: the pose partials
    live in the library's static device array (for callers that cannot
    allocate device memory). grads.grad2d is the input; grads.pose_partials
    is not used."""
    _check(load().gs_project_bwd_noalloc(ctypes.byref(g.c()), ctypes.byref(views.c()), ctypes.byref(cfg),
                                         _ptr(proj), _ptr(grads.grad2d), ctypes.byref(grads.c()),
                                         int(bool(want_gaussian_grads)), _ptr(dL_dviewmat), _ptr(dL_dtwist),
                                         _ptr(status), _stream(stream)), "gs_project_bwd_noalloc")


def gs_sgld_adam_step(groups, step, beta1=0.9, beta2=0.999, eps=1e-15, noise=None, noise_scale=0.0, noise_group=0,
                      stream=None):
    """Eq. 1 update in one launch. groups: list of (param, grad, exp_avg,
    exp_avg_sq, lr) CUDA float32 tensors (updated in place)."""
    arr = (gs_adam_group * len(groups))()
    for k, (p, g, m, v, lr) in enumerate(groups):
        assert p.numel() == g.numel() == m.numel() == v.numel()
        arr[k] = gs_adam_group(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), float(lr))
    _check(load().gs_sgld_adam_step(arr, len(groups), int(step), ctypes.c_double(beta1), ctypes.c_double(beta2),
                                    ctypes.c_double(eps), _ptr(noise), ctypes.c_float(noise_scale), int(noise_group),
                                    _stream(stream)), "gs_sgld_adam_step")


# ---------------------------------------------------------------------------
# camera global alignment (Section 3.3)
# ---------------------------------------------------------------------------
def gs_ga_select_pairs(viewmats, max_angle_deg, pairs, n_pairs_out, status=None, stream=None):
    """Candidate pairs into pairs (int32 [capacity,2]); count into
    n_pairs_out (int64 [1])."""
    cap = pairs.shape[0] if pairs is not None else 0
    _check(load().gs_ga_select_pairs(_ptr(viewmats), int(viewmats.shape[0]), ctypes.c_double(max_angle_deg),
                                     _ptr(pairs) if cap else None, ctypes.c_int64(cap), _ptr(n_pairs_out),
                                     _ptr(status), _stream(stream)), "gs_ga_select_pairs")


def gs_ga_incidence(pairs, n_cams, cam_offsets, cam_pairs, status=None, stream=None):
    _check(load().gs_ga_incidence(_ptr(pairs) if pairs.numel() else None, ctypes.c_int64(pairs.shape[0]),
                                  int(n_cams), _ptr(cam_offsets), _ptr(cam_pairs) if cam_pairs.numel() else None,
                                  _ptr(status), _stream(stream)), "gs_ga_incidence")


def ga_problem(intrinsics, viewmats, pairs, match_offsets, matches, weights=None) -> gs_ga_problem:
    return gs_ga_problem(int(intrinsics.shape[0]), _ptr(intrinsics), _ptr(viewmats), int(pairs.shape[0]),
                         _ptr(pairs) if pairs.numel() else None, _ptr(match_offsets), int(matches.shape[0]),
                         _ptr(matches) if matches.numel() else None, _ptr(weights))


def gs_ga_epipolar(problem: gs_ga_problem, pair_sums, loss, dist=None, cam_offsets=None, cam_pairs=None,
                   d_intrinsics=None, d_viewmats=None, status=None, stream=None):
    _check(load().gs_ga_epipolar(ctypes.byref(problem), _ptr(dist),
                                 _ptr(pair_sums) if pair_sums is not None and pair_sums.numel() else None,
                                 _ptr(cam_offsets), _ptr(cam_pairs) if cam_pairs is not None and cam_pairs.numel()
                                 else None, _ptr(loss), _ptr(d_intrinsics), _ptr(d_viewmats), _ptr(status),
                                 _stream(stream)), "gs_ga_epipolar")


def ga_state(intrinsics0, viewmats0, residuals, exp_avg, exp_avg_sq, step, intrinsics, viewmats, lr, beta1=0.9,
             beta2=0.999, eps=1e-15, optimise_focal=True) -> gs_ga_state:
    return gs_ga_state(int(intrinsics0.shape[0]), _ptr(intrinsics0), _ptr(viewmats0), _ptr(residuals),
                       _ptr(exp_avg), _ptr(exp_avg_sq), _ptr(step), _ptr(intrinsics), _ptr(viewmats), float(lr),
                       float(beta1), float(beta2), float(eps), int(bool(optimise_focal)))


def gs_ga_step(state: gs_ga_state, problem: gs_ga_problem, pair_sums, cam_offsets, cam_pairs, loss,
               d_residuals=None, status=None, stream=None):
    _check(load().gs_ga_step(ctypes.byref(state), ctypes.byref(problem),
                             _ptr(pair_sums) if pair_sums.numel() else None, _ptr(cam_offsets),
                             _ptr(cam_pairs) if cam_pairs.numel() else None, _ptr(loss), _ptr(d_residuals),
                             _ptr(status), _stream(stream)), "gs_ga_step")


def gs_ga_weights_scratch_bytes(n_bins):
    return int(load().gs_ga_weights_scratch_bytes(int(n_bins)))


def gs_ga_weights(dist, n_bins, alpha, counts, weights, stats, scratch, stream=None):
    n = dist.numel()
    _check(load().gs_ga_weights(_ptr(dist) if n else None, ctypes.c_int64(n), int(n_bins), ctypes.c_double(alpha),
                                _ptr(counts), _ptr(weights) if n else None, _ptr(stats), _ptr(scratch),
                                _stream(stream)), "gs_ga_weights")


def pair_counts(bins: Bins):
    """(fwd evaluated, fwd composited, bwd evaluated, bwd composited) pixel-
    Gaussian pairs of the last render calls (reads the device counters; the
    backward counts only when its config has count_pairs set)."""
    c = bins.counters.cpu().numpy().view(np.int64)
    return int(c[4]), int(c[5]), int(c[6]), int(c[7])


def gs_pose_grad(views: Views, pose_partials, n_blocks, dL_dviewmat, dL_dtwist=None, stream=None):
    _check(load().gs_pose_grad(ctypes.byref(views.c()), _ptr(pose_partials), int(n_blocks), _ptr(dL_dviewmat),
                               _ptr(dL_dtwist), _stream(stream)), "gs_pose_grad")


def gs_l1_dssim_loss(views: Views, image, target, loss, dL_dimage, lam=0.2, stream=None):
    """L1 + D-SSIM loss (loss [3] = total, mean L1, 1 - mean SSIM) and its
    gradient, views concatenated [3,H,W] each."""
    _check(load().gs_l1_dssim_loss(ctypes.byref(views.c()), _ptr(image), _ptr(target), ctypes.c_float(lam),
                                   _ptr(loss), _ptr(dL_dimage), _stream(stream)), "gs_l1_dssim_loss")


def gs_workspace_size(views: Views, cfg: gs_config, n_gaussians, capacity):
    """Bytes of the one-buffer step workspace (tile lists, 2D gradients, pose
    partials); host arithmetic only."""
    return int(load().gs_workspace_size(ctypes.byref(views.c()), ctypes.byref(cfg), int(n_gaussians),
                                        int(capacity)))


def gs_workspace_carve(views: Views, cfg: gs_config, n_gaussians, capacity, ws_ptr, ws_bytes):
    """(gs_bins, grad2d address, pose_partials address) carved from the
    workspace at device address ws_ptr (host arithmetic only)."""
    b = gs_bins()
    gr = gs_grads()
    _check(load().gs_workspace_carve(ctypes.byref(views.c()), ctypes.byref(cfg), int(n_gaussians), int(capacity),
                                     ctypes.c_void_p(ws_ptr), ctypes.c_size_t(ws_bytes), ctypes.byref(b),
                                     ctypes.byref(gr)), "gs_workspace_carve")
    return b, gr.grad2d, gr.pose_partials


def gs_status_read(status, stream=None):
    """The device status word as 4 host ints, after the stream's work so far
    (the library's one synchronising call)."""
    out = (ctypes.c_int32 * 4)()
    _check(load().gs_status_read(_ptr(status), out, _stream(stream)), "gs_status_read")
    return list(out)


def gs_spatial_codes(means, box, codes, stream=None):
    """Morton codes (int64 tensor viewed as uint64) of means [n,3] in box
    (six floats: lo xyz, hi xyz)."""
    b = (ctypes.c_float * 6)(*[float(v) for v in box])
    _check(load().gs_spatial_codes(_ptr(means) if means.numel() else None, ctypes.c_int64(means.shape[0]), b,
                                   _ptr(codes) if codes.numel() else None, _stream(stream)), "gs_spatial_codes")


def gs_peak_probe(kind, iters, out=None, stream=None):
    """One launch of the arithmetic-throughput probe (kind 0 FP32 FMA, 1
    packed f32x2 FMA, 2 ex2.approx); returns (out, operations per launch,
    counting an FMA lane as one operation)."""
    blocks = int(load().gs_probe_blocks())
    if out is None:
        out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    _check(load().gs_peak_probe(int(kind), int(iters), _ptr(out), _stream(stream)), "gs_peak_probe")
    return out, blocks * 256 * 8 * int(iters) * (2 if kind == 1 else 1)


def gs_check_bounded_wait(status, stream=None):
    """Enqueue the bounded-wait check: status (int32[4], zeroed by the
    caller) becomes {GS_ERR_TIMEOUT, 0, ...} after about a second."""
    _check(load().gs_check_bounded_wait(_ptr(status), _stream(stream)), "gs_check_bounded_wait")


def gs_l1_loss(image, target, loss, dL_dimage, stream=None):
    _check(load().gs_l1_loss(_ptr(image), _ptr(target), ctypes.c_int64(image.numel()), _ptr(loss),
                             _ptr(dL_dimage), _stream(stream)), "gs_l1_loss")
