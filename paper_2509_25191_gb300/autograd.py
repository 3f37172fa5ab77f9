"""torch.autograd wrapper and buffer/capacity management over the C ABI.

``Rasterizer`` owns the device buffers of one views layout (projected
records, tile lists, gradient scratch) and plans the tile-instance capacity:
uncaptured calls read the instance count back once per forward (4 bytes) and
grow the buffers when needed; captured (CUDA graph) calls run with a fixed
capacity and report overflow through the device status word.

``RasterizeViews`` is the autograd.Function: forward = gs_project +
gs_bin_sort + gs_render_fwd, backward = gs_render_bwd + gs_pose_grad (after
rebuilding the forward's tile lists if the same ``Rasterizer`` has run
another forward in between). The
backward recomputes transmittance from the forward image instead of storing
it (Section 3.4's joint pose optimisation over many views needs the memory).
Gradients flow to means, log-scales, quaternions, opacity logits, SH
coefficients and the world->camera view matrices [V,12]; the pose residuals
(``pose.py``) chain from there with ordinary torch ops.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import _lib
from ._lib import Bins, Gaussians, Grads, Views

INSTANCE_LIMIT = 0x7fffffff   # the instance count saturates here (32-bit tile ranges)


class Rasterizer:
    def __init__(self, tile=(16, 16), pixel_gate=True, bg=(0.0, 0.0, 0.0), capacity_headroom=1.3, **kw):
        self.cfg = _lib.config(tile=tile, pixel_gate=pixel_gate, bg=bg, **kw)
        self.tile = tuple(tile)
        self.headroom = float(capacity_headroom)
        self.bins = None
        self.status = None
        self.fixed_capacity = False   # set for graph capture: never read back
        self._grads = None
        self.last_instances = None
        self.generation = 0           # counts bin_sort calls: which forward the tile lists belong to

    # ------------------------------------------------------------------
    def _ensure_bins(self, views: Views, capacity: int, device):
        T = views.num_tiles(self.cfg)
        if (self.bins is None or self.bins.n_tiles != T or self.bins.capacity < capacity or
                self.bins.pixels != views.pixels):
            self.bins = Bins(T, capacity, device, pixels=views.pixels)
        if self.status is None or self.status.device != torch.device(device):
            self.status = _lib.new_status(device)
        return self.bins

    def reserve(self, views: Views, capacity: int, device="cuda"):
        """Fix the instance capacity (for CUDA-graph capture)."""
        self.bins = None
        self._ensure_bins(views, int(capacity), device)
        self.fixed_capacity = True

    def project(self, g: Gaussians, views: Views, proj=None):
        if proj is None:
            proj = torch.empty(max(1, views.num_slots()), _lib.GS_RECORD_FLOATS, dtype=torch.float32,
                               device=g.means.device)
        _lib.gs_project(g, views, self.cfg, proj, self.status)
        return proj

    def bin_sort(self, views: Views, proj):
        dev = proj.device
        if self.bins is None:
            self._ensure_bins(views, max(1024, 4 * views.num_slots()), dev)
        elif self.bins.n_tiles != views.num_tiles(self.cfg) or self.bins.pixels != views.pixels:
            self._ensure_bins(views, self.bins.capacity, dev)
        _lib.gs_bin_sort(views, self.cfg, proj, self.bins, self.status)
        self.generation += 1
        if not self.fixed_capacity:
            n = int(self.bins.counters[0].item())   # the one readback of the uncaptured path
            self.last_instances = n
            if n >= INSTANCE_LIMIT:
                # the count saturates at 2^31 - 1: more instances than the
                # 32-bit tile ranges can address; growing cannot help
                raise _lib.GsError(_lib.GS_ERR_OVERFLOW, f"gs_bin_sort ({n} or more tile instances)")
            if n > self.bins.capacity:
                self.status.zero_()
                self._ensure_bins(views, int(math.ceil(n * self.headroom)) + 1024, dev)
                _lib.gs_bin_sort(views, self.cfg, proj, self.bins, self.status)
                self.check_status()   # the re-bin must fit (it reads the status word once)
        return self.bins

    def render(self, views: Views, proj, bins: Bins, image=None):
        if image is None:
            image = torch.empty(views.num_image_floats(), dtype=torch.float32, device=proj.device)
        _lib.gs_render_fwd(views, self.cfg, proj, bins, image, self.status)
        return image

    def forward(self, g: Gaussians, views: Views):
        proj = self.project(g, views)
        bins = self.bin_sort(views, proj)
        image = self.render(views, proj, bins)
        return image, proj

    def grads_buffers(self, g: Gaussians, views: Views, want_gaussian_grads=True):
        key = (g.n, g.sh_degree, views.num_slots(), views.n, want_gaussian_grads, g.means.device)
        if self._grads is None or self._grads[0] != key:
            self._grads = (key, Grads(g.n, g.sh_degree, views.num_slots(), views.n, g.means.device,
                                      want_gaussian_grads))
        return self._grads[1]

    def backward(self, g: Gaussians, views: Views, proj, image, dL_dimage, want_gaussian_grads=True,
                 grads: Grads = None, use_last=True):
        """use_last=False when the tile lists were rebuilt after another
        forward wrote the last-contributor record (the replay then runs to
        saturation instead; the same gradients)."""
        grads = grads or self.grads_buffers(g, views, want_gaussian_grads)
        _lib.gs_render_bwd(g, views, self.cfg, proj, self.bins, image, dL_dimage, grads, want_gaussian_grads,
                           self.status, use_last=use_last)
        dvm = torch.empty(views.n, 12, dtype=torch.float32, device=proj.device)
        dtw = torch.empty(views.n, 6, dtype=torch.float32, device=proj.device)
        _lib.gs_pose_grad(views, grads.pose_partials, grads.n_blocks, dvm, dtw)
        return grads, dvm, dtw

    def backward_l1(self, g: Gaussians, views: Views, proj, image, target, loss, want_gaussian_grads=True,
                    grads: Grads = None, use_last=True):
        """The backward of the mean L1 loss against target, with the loss
        folded into the raster backward (loss[0] = mean |image - target|;
        no dL/dimage buffer)."""
        grads = grads or self.grads_buffers(g, views, want_gaussian_grads)
        _lib.gs_rasterize_bwd_l1(views, self.cfg, proj, self.bins, image, target, loss, grads.grad2d, self.status,
                                 use_last=use_last)
        _lib.gs_project_bwd(g, views, self.cfg, proj, grads, want_gaussian_grads, self.status)
        dvm = torch.empty(views.n, 12, dtype=torch.float32, device=proj.device)
        dtw = torch.empty(views.n, 6, dtype=torch.float32, device=proj.device)
        _lib.gs_pose_grad(views, grads.pose_partials, grads.n_blocks, dvm, dtw)
        return grads, dvm, dtw

    def check_status(self):
        """Read the device status word (synchronises); raise on a device error."""
        st = self.status.cpu().numpy()
        if st[0] != 0:
            needed = int(st[1]) & 0xffffffff | (int(st[2]) << 32)
            raise _lib.GsError(int(st[0]), f"device status (instances needed: {needed})")


class RasterizeViews(torch.autograd.Function):
    """images = RasterizeViews.apply(means, log_scales, quats, opacity_logits,
    sh, viewmats, intrinsics, layout, rasterizer); images is the flat
    concatenation of the views' [3,H,W] images."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, viewmats, intrinsics, layout, rast):
        g = Gaussians(means.detach().contiguous(), log_scales.detach().contiguous(), quats.detach().contiguous(),
                      opacity_logits.detach().contiguous(), sh.detach().contiguous())
        views = Views(viewmats.detach().contiguous(), intrinsics.detach().contiguous(), *layout)
        image, proj = rast.forward(g, views)
        ctx.rast, ctx.g, ctx.views, ctx.proj, ctx.generation = rast, g, views, proj, rast.generation
        ctx.want_gauss = any(ctx.needs_input_grad[:5])
        ctx.save_for_backward(image)
        return image

    @staticmethod
    def backward(ctx, dL_dimage):
        (image,) = ctx.saved_tensors
        own = ctx.rast.generation == ctx.generation
        if not own:
            # the rasterizer has binned another forward since: rebuild this
            # forward's tile lists from its projected records (same lists);
            # the last-contributor record is the other forward's, so the
            # replay runs without it
            ctx.rast.bin_sort(ctx.views, ctx.proj)
        grads, dvm, _ = ctx.rast.backward(ctx.g, ctx.views, ctx.proj, image, dL_dimage.contiguous(),
                                          want_gaussian_grads=ctx.want_gauss, use_last=own)
        if ctx.want_gauss:
            out = [grads.means.clone(), grads.log_scales.clone(), grads.quats.clone(),
                   grads.opacity_logits.clone(), grads.sh.clone()]
        else:
            out = [None] * 5
        return (*out, dvm, None, None, None)


def rasterize(means, log_scales, quats, opacity_logits, sh, viewmats, intrinsics, width, height,
              gauss_begin=None, gauss_count=None, rasterizer: Rasterizer = None):
    """Differentiable render of V views; returns the flat image tensor."""
    V = viewmats.shape[0]
    n = means.shape[0]
    gauss_begin = np.zeros(V, np.int64) if gauss_begin is None else gauss_begin
    gauss_count = np.full(V, n, np.int64) if gauss_count is None else gauss_count
    layout = (np.asarray(width, np.int32), np.asarray(height, np.int32), np.asarray(gauss_begin, np.int64),
              np.asarray(gauss_count, np.int64))
    rasterizer = rasterizer or Rasterizer()
    return RasterizeViews.apply(means, log_scales, quats, opacity_logits, sh, viewmats, intrinsics, layout,
                                rasterizer)


def split_views(image, width, height):
    """Flat image -> list of [3,H,W] views (no copy)."""
    out, off = [], 0
    for W, H in zip(width, height):
        n = 3 * int(W) * int(H)
        out.append(image[off:off + n].view(3, int(H), int(W)))
        off += n
    return out
