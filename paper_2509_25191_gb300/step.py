"""One training step of the rasterizer, captured as a CUDA graph.

A step over a batch of views is: gs_project -> gs_bin_sort -> gs_render_fwd
-> gs_rasterize_bwd_l1 (the mean L1 loss against the step's target images,
folded into the raster backward) or gs_l1_dssim_loss -> gs_rasterize_bwd ->
gs_project_bwd -> gs_pose_grad, i.e. the photometric supervision of
Section 3.1 with gradients to every Gaussian parameter and to every view's
pose (Section 3.4). All buffers are allocated once; the tile-instance
capacity is sized from one uncaptured forward (with headroom) and the step is
captured into a CUDA graph, so replaying it launches every kernel with no
host synchronisation. New inputs (Gaussian parameters, view matrices,
targets) are copied into the captured tensors before a replay; an instance
count above the capacity is reported in the device status word and
``GraphStep.check()`` re-plans.

With ``slots=2`` the step keeps two copies of its per-step inputs (target
images and view matrices, and with ``slot_gaussians=True`` the Gaussian
parameters too) and of its results (``loss_slots``, ``dviewmat_slots``,
``dtwist_slots``; ``loss`` and ``dviewmat`` are slot 0's) and captures one
graph per slot, sharing every other buffer:
a training loop writes step k+1's inputs into the other slot (e.g. by an
asynchronous host-to-device copy on another stream) while step k runs, and
replays ``replay(k % 2)``. Gaussian slots are separate tensors (slot 0 is
the caller's, slot 1 starts as a copy): an in-place update of one slot's
parameters does not reach the other, so a loop that updates the parameters
on the device writes each step's parameters into the slot it replays.

``PlainStep`` is the uncaptured reference path: the same calls made view by
view, each with the host readback of the instance count that an uncaptured
call needs.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib
from ._lib import Gaussians, Grads, Views
from .autograd import Rasterizer


class GraphStep:
    # project 1, bin/sort 5 (count, scan, scatter, split, sort), render 1, the
    # zeroing of the backward's accumulators 1 (a kernel with overlap_prev),
    # raster bwd 1, projection bwd 1, pose 1; the L1 loss is part of the raster
    # backward, the L1 + D-SSIM loss adds 2 kernels
    KERNELS_FIXED = 11
    # the calls of a step, in order (the stages of run()'s events)
    STAGES = {"l1": ("gs_project", "gs_bin_sort", "gs_render_fwd", "gs_rasterize_bwd_l1", "gs_project_bwd",
                     "gs_pose_grad"),
              "l1_dssim": ("gs_project", "gs_bin_sort", "gs_render_fwd", "gs_l1_dssim_loss", "gs_rasterize_bwd",
                           "gs_project_bwd", "gs_pose_grad")}

    @property
    def stages(self):
        return self.STAGES[self.loss_kind]

    def kernels_per_step(self) -> int:
        """Kernels of this library that one step launches: the fixed eleven, the
        D-SSIM loss kernels, and, when the image has fewer than 16 tiles per
        SM, the tile orderings by replay length that the raster forward (from
        the previous forward's record) and the raster backward run first."""
        loss = 0 if self.loss_kind == "l1" else 2
        sms = torch.cuda.get_device_properties(self.g.means.device).multi_processor_count
        order = 2 if 0 < self.bins.n_tiles < 16 * sms else 0
        return self.KERNELS_FIXED + loss + order

    def __init__(self, g: Gaussians, views: Views, target, tile=(16, 16), headroom=1.25, capture=True,
                 want_gaussian_grads=True, loss="l1", lam=0.2, slots=1, slot_gaussians=False, capacity=None,
                 batch=(2, 1)):
        self.g, self.views, self.target = g, views, target
        if slots < 1:
            raise ValueError("slots must be >= 1")
        # per-slot inputs: slot 0 is the caller's target and view matrices
        self.target_slots = [target] + [torch.empty_like(target) for _ in range(slots - 1)]
        self.viewmat_slots = [views.viewmats] + [torch.empty_like(views.viewmats) for _ in range(slots - 1)]
        self.slot_views = [views] + [Views(vm, views.intrinsics, views.width, views.height, views.gauss_begin,
                                           views.gauss_count) for vm in self.viewmat_slots[1:]]
        # (a Gaussian slot starts as a copy of the caller's parameters)
        self.gauss_slots = [g] + [Gaussians(*(t.clone() for t in (g.means, g.log_scales, g.quats,
                                                                  g.opacity_logits, g.sh)))
                                  if slot_gaussians else g for _ in range(slots - 1)]
        self.want = want_gaussian_grads
        if loss not in ("l1", "l1_dssim"):
            raise ValueError(f"unknown loss {loss!r}")
        self.loss_kind, self.lam = loss, float(lam)
        dev = g.means.device
        # the step's calls run in a fixed order, so the backward's zeroing may
        # overlap the tail of the kernel ahead (gs_config.overlap_prev)
        self.rast = Rasterizer(tile=tile, batch=batch, overlap_prev=True)
        if capacity is None:
            # size the instance capacity from one uncaptured forward
            _, _ = self.rast.forward(g, views)
            torch.cuda.synchronize(dev)
            capacity = int(self.rast.last_instances * headroom) + 4096
        self.capacity = int(capacity)
        self.rast.reserve(views, self.capacity, dev)
        self.cfg, self.bins, self.status = self.rast.cfg, self.rast.bins, self.rast.status
        self.proj = torch.empty(max(1, views.num_slots()), _lib.GS_RECORD_FLOATS, device=dev)
        self.image = torch.empty(views.num_image_floats(), device=dev)
        # dL/dimage of the L1 + D-SSIM loss (the L1 loss forms its own in the raster backward)
        self.dimg = torch.empty_like(self.image) if loss == "l1_dssim" else None
        # l1: [mean L1]; l1_dssim: [total, mean L1, 1 - mean SSIM]
        # the step's results (loss, pose gradient) are kept per input slot, so
        # that a loop can read step k's back while step k+1 runs
        self.loss_slots = [torch.empty(1 if loss == "l1" else 3, device=dev) for _ in range(slots)]
        self.loss = self.loss_slots[0]
        self.grads = Grads(g.n, g.sh_degree, views.num_slots(), views.n, dev, want_gaussian_grads)
        self.dviewmat_slots = [torch.empty(views.n, 12, device=dev) for _ in range(slots)]
        self.dtwist_slots = [torch.empty(views.n, 6, device=dev) for _ in range(slots)]
        self.dviewmat, self.dtwist = self.dviewmat_slots[0], self.dtwist_slots[0]
        self.graph = None
        self.graphs = []
        if capture:
            self.capture()

    def run(self, events=None, slot=0):
        """Enqueue the step on the current stream (optionally recording an
        event before and after every call), reading the inputs of ``slot``."""
        rec = (lambda: events.append(torch.cuda.Event(enable_timing=True)) or events[-1].record()) \
            if events is not None else (lambda: None)
        g, v, cfg, b, st = self.gauss_slots[slot], self.slot_views[slot], self.cfg, self.bins, self.status
        target = self.target_slots[slot]
        rec()
        _lib.gs_project(g, v, cfg, self.proj, st)
        rec()
        _lib.gs_bin_sort(v, cfg, self.proj, b, st)
        rec()
        _lib.gs_render_fwd(v, cfg, self.proj, b, self.image, st)
        rec()
        if self.loss_kind == "l1":
            _lib.gs_rasterize_bwd_l1(v, cfg, self.proj, b, self.image, target, self.loss_slots[slot],
                                     self.grads.grad2d, st)
            rec()
        else:
            _lib.gs_l1_dssim_loss(v, self.image, target, self.loss_slots[slot], self.dimg, self.lam)
            rec()
            _lib.gs_rasterize_bwd(v, cfg, self.proj, b, self.image, self.dimg, self.grads.grad2d, st)
            rec()
        _lib.gs_project_bwd(g, v, cfg, self.proj, self.grads, self.want, st)
        rec()
        _lib.gs_pose_grad(v, self.grads.pose_partials, self.grads.n_blocks, self.dviewmat_slots[slot],
                          self.dtwist_slots[slot])
        rec()

    def capture(self):
        dev = self.g.means.device
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        self.graphs = []
        with torch.cuda.stream(s):
            self.run()
            torch.cuda.synchronize(dev)
            for slot in range(len(self.target_slots)):
                gr = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gr, stream=s):
                    self.run(slot=slot)
                self.graphs.append(gr)
        torch.cuda.synchronize(dev)
        self.graph = self.graphs[0]

    def replay(self, slot=0):
        self.graphs[slot].replay()

    def check(self):
        """Read the status word (synchronises). On a capacity overflow, grow
        the capacity, clear the word, re-capture, and report True (the step
        must be rerun); otherwise report False. A loop of the form
        ``while step.check(): step.replay()`` ends after the first replay
        that fits."""
        st = self.status.cpu().numpy()
        if st[0] == 0:
            return False
        if st[0] != _lib.GS_ERR_CAPACITY:
            raise _lib.GsError(int(st[0]), "device status")
        needed = (int(st[1]) & 0xffffffff) | (int(st[2]) << 32)
        self.capacity = int(needed * 1.25) + 4096
        self.rast.reserve(self.views, self.capacity, self.g.means.device)
        self.bins, self.status = self.rast.bins, self.rast.status
        # the overflow has been handled: clear the word (no kernel resets it),
        # so that the next check reports only what the next replay finds
        self.status.zero_()
        self.capture()
        return True


class PlainStep:
    """The same step, uncaptured and view by view."""

    def __init__(self, g: Gaussians, views: Views, target, tile=(16, 16), batch=(2, 1)):
        self.g = g
        self.one = []
        off = 0
        for v in range(views.n):
            vv = Views(views.viewmats[v:v + 1], views.intrinsics[v:v + 1], views.width[v:v + 1],
                       views.height[v:v + 1], views.gauss_begin[v:v + 1], views.gauss_count[v:v + 1])
            n = vv.num_image_floats()
            self.one.append((vv, target[off:off + n], Rasterizer(tile=tile, batch=batch, overlap_prev=True)))
            off += n
        dev = g.means.device
        self.loss = torch.empty(1, device=dev)

    STAGES = ("project", "bin_sort", "render_fwd", "backward_l1")

    def run(self, events=None):
        """The views one after another; with ``events`` (a list), an event is
        recorded before and after each stage of each view (the bin_sort stage
        includes the instance-count readback)."""
        rec = (lambda: events.append(torch.cuda.Event(enable_timing=True)) or events[-1].record()) \
            if events is not None else (lambda: None)
        for vv, tgt, rast in self.one:
            rec()
            proj = rast.project(self.g, vv)
            rec()
            bins = rast.bin_sort(vv, proj)                 # includes the instance-count readback
            rec()
            image = rast.render(vv, proj, bins)
            rec()
            rast.backward_l1(self.g, vv, proj, image, tgt, self.loss)
            rec()
