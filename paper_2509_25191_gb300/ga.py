"""Camera global alignment (Section 3.3, Eqs. 2-4) on the GPU.

Given initial cameras (intrinsics, world-to-camera extrinsics) and keypoint
matches for image pairs, refine every camera by minimising the weighted
epipolar distance of Eq. 2. The weights of Eq. 3 and the learning rate of
Eq. 4 are fixed once from the distances under the initial cameras; then
``iterations`` (300 in Section 4.1) Adam steps move per-camera residuals:
the 6D rotation residual and translation residual of Section 3.4 (R' = dR R,
t' = t + dt) and a log-focal residual (f' = f exp(df)). By default an
iteration is one gs_ga_step call: three kernels (cameras from the residuals;
distances and per-pair gradient sums; per-camera reduction, chain to the
residuals and Adam) with no host work. ``fused=False`` runs the same
iteration as gs_ga_epipolar, the residual ops in torch with autograd, and
gs_sgld_adam_step.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib, pose

LRS = (5e-4, 1e-3, 1e-2)      # lr0, lr1, lr2 (Section 4.1)
BOUNDS = (2.5, 7.5)           # b1, b2 in pixels (Section 4.1)


def lr_rule(median, lrs=LRS, bounds=BOUNDS):
    """Eq. 4: lr0 below b1, lr2 above b2, lr1 in between (inclusive)."""
    if median < bounds[0]:
        return lrs[0]
    if median > bounds[1]:
        return lrs[2]
    return lrs[1]


def select_pairs(viewmats, max_angle_deg=30.0, capacity=None):
    """Candidate pairs (int32 [M,2], row-major i < j) of cameras whose viewing
    directions are less than ``max_angle_deg`` apart. Reads the count back
    (one synchronisation)."""
    n = viewmats.shape[0]
    dev = viewmats.device
    cap = n * (n - 1) // 2 if capacity is None else int(capacity)
    pairs = torch.empty(max(cap, 1), 2, dtype=torch.int32, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    status = _lib.new_status(dev)
    _lib.gs_ga_select_pairs(viewmats.contiguous(), max_angle_deg, pairs[:cap], count, status)
    st = status.cpu().numpy()
    if st[0] != 0:
        raise _lib.GsError(int(st[0]), f"gs_ga_select_pairs ({int(count.item())} pairs found)")
    return pairs[:int(count.item())].contiguous()


def incidence(pairs, n_cams):
    dev = pairs.device
    offs = torch.empty(n_cams + 1, dtype=torch.int32, device=dev)
    lists = torch.empty(max(1, 2 * pairs.shape[0]), dtype=torch.int32, device=dev)
    status = _lib.new_status(dev)
    _lib.gs_ga_incidence(pairs, n_cams, offs, lists[:2 * pairs.shape[0]], status)
    return offs, lists[:2 * pairs.shape[0]], status


def pdf_weights(dist, n_bins=100, alpha=0.5):
    """Eq. 3 weights of the distances, the histogram counts and the stats
    {max, lower middle, upper middle, 0} (device tensors, no host read)."""
    dev = dist.device
    n = dist.numel()
    w = torch.empty(n, dtype=torch.float32, device=dev)
    counts = torch.empty(n_bins, dtype=torch.int32, device=dev)
    stats = torch.empty(4, dtype=torch.float32, device=dev)
    scratch = torch.empty(_lib.gs_ga_weights_scratch_bytes(n_bins) // 4, dtype=torch.int32, device=dev)
    _lib.gs_ga_weights(dist, n_bins, alpha, counts, w, stats, scratch)
    return w, counts, stats


class GlobalAlignment:
    """One global-alignment problem resident on the GPU."""

    def __init__(self, intrinsics, viewmats, pairs, match_offsets, matches, n_bins=100, alpha=0.5, lrs=LRS,
                 bounds=BOUNDS, optimise_focal=True, fused=True):
        dev = viewmats.device
        self.n = int(viewmats.shape[0])
        self.intr0 = intrinsics.detach().float().contiguous()
        self.vm0 = viewmats.detach().float().contiguous()
        self.pairs = pairs.contiguous()
        self.offsets = match_offsets.contiguous()
        self.matches = matches.contiguous()
        self.cam_offsets, self.cam_pairs, self.status = incidence(self.pairs, self.n)
        self.pair_sums = torch.empty(max(1, self.pairs.shape[0]), _lib.GS_GA_PAIR_FLOATS, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.d_intr = torch.empty(self.n, 4, device=dev)
        self.d_vm = torch.empty(self.n, 12, device=dev)
        # Eq. 3 weights and the Eq. 4 learning rate from the initial distances
        self.dist0 = torch.empty(self.matches.shape[0], device=dev)
        prob = _lib.ga_problem(self.intr0, self.vm0, self.pairs, self.offsets, self.matches)
        _lib.gs_ga_epipolar(prob, self.pair_sums, self.loss, dist=self.dist0, status=self.status)
        self.weights, self.counts, stats = pdf_weights(self.dist0, n_bins, alpha)
        st = stats.cpu().numpy().astype(np.float64)
        self.median0 = 0.5 * (st[1] + st[2])
        self.lr = lr_rule(self.median0, lrs, bounds)
        self.optimise_focal = optimise_focal
        # residual parameters and their Adam moments
        self.dr = pose.identity_6d(self.n, device=dev)
        self.dt = torch.zeros(self.n, 3, device=dev)
        self.dlogf = torch.zeros(self.n, 1, device=dev)
        self.params = [self.dr, self.dt] + ([self.dlogf] if optimise_focal else [])
        self.moments = [(torch.zeros_like(p), torch.zeros_like(p)) for p in self.params]
        self.steps = 0
        # fused state: residuals [N,10] = (6D rotation, translation, log focal)
        self.fused = fused
        self.res = torch.cat([self.dr, self.dt, self.dlogf], 1).contiguous()
        self.res_m = torch.zeros_like(self.res)
        self.res_v = torch.zeros_like(self.res)
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        self.intr = self.intr0.clone()
        self.vm = self.vm0.clone()
        self.state = _lib.ga_state(self.intr0, self.vm0, self.res, self.res_m, self.res_v, self.step_dev, self.intr,
                                   self.vm, self.lr, optimise_focal=optimise_focal)
        self.fused_problem = _lib.ga_problem(self.intr, self.vm, self.pairs, self.offsets, self.matches, self.weights)

    def cameras(self, params=None):
        if params is None and self.fused:
            params = (self.res[:, :6], self.res[:, 6:9], self.res[:, 9:10])
        dr, dt, dlogf = params if params is not None else (self.dr, self.dt, self.dlogf)
        vm = pose.apply_residual(self.vm0, dr, dt)
        intr = torch.cat([self.intr0[:, :2] * torch.exp(dlogf), self.intr0[:, 2:]], 1)
        return intr, vm

    def problem(self, intr, vm):
        return _lib.ga_problem(intr, vm, self.pairs, self.offsets, self.matches, self.weights)

    def loss_and_grads(self, intr, vm):
        """Eq. 2 loss and dL/d(intrinsics), dL/d(viewmats) at the given cameras."""
        _lib.gs_ga_epipolar(self.problem(intr.contiguous(), vm.contiguous()), self.pair_sums, self.loss,
                            cam_offsets=self.cam_offsets, cam_pairs=self.cam_pairs, d_intrinsics=self.d_intr,
                            d_viewmats=self.d_vm, status=self.status)
        return self.loss, self.d_intr, self.d_vm

    def step(self, d_residuals=None):
        if self.fused:
            _lib.gs_ga_step(self.state, self.fused_problem, self.pair_sums, self.cam_offsets, self.cam_pairs,
                            self.loss, d_residuals, self.status)
            self.steps += 1
            return self.loss
        leaves = [self.dr.detach().requires_grad_(True), self.dt.detach().requires_grad_(True),
                  self.dlogf.detach().requires_grad_(self.optimise_focal)]
        with torch.enable_grad():
            intr, vm = self.cameras(leaves)
        self.loss_and_grads(intr.detach(), vm.detach())
        outs, gouts = [vm], [self.d_vm]
        if self.optimise_focal:
            outs.append(intr)
            gouts.append(self.d_intr)
        grads = torch.autograd.grad(outs, leaves[:len(self.params)], gouts)
        self.steps += 1
        _lib.gs_sgld_adam_step([(p, g.contiguous(), m, v, self.lr)
                                for p, g, (m, v) in zip(self.params, grads, self.moments)], self.steps)
        return self.loss

    def run(self, iterations=300):
        for _ in range(iterations):
            self.step()
        return self.cameras()

    def check(self):
        st = self.status.cpu().numpy()
        if st[0] != 0:
            raise _lib.GsError(int(st[0]), f"global alignment (detail {int(st[1])})")
