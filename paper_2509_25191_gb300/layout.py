"""Spatial order of the Gaussians (data layout for training loops).

No result of the rasterizer depends on the order of the Gaussians (images
and gradients are permutation-invariant for distinct depths; equal depths
are ordered by index). A training loop may therefore keep its Gaussians
sorted along a Morton curve of their means, refreshed whenever it adds or
removes Gaussians: Gaussians that project near each other are then
neighbours in memory, so binning blocks write longer runs per tile and the
projection backward's warps agree on which Gaussians carry a gradient. The
codes come from the library's kernel (gs_spatial_codes); the sort and the
gather of the parameter tensors are torch's.
"""
from __future__ import annotations

import torch

from . import _lib
from ._lib import Gaussians


def spatial_order(means: torch.Tensor, ranges=None) -> torch.Tensor:
    """Permutation (int64, on the means' device) that sorts each range
    (begin, count) of means -- one per scene; the whole array by default --
    by Morton code in that range's bounding box, leaving every Gaussian in
    its range; the identity outside the ranges."""
    n = means.shape[0]
    perm = torch.arange(n, device=means.device)
    for begin, count in (ranges if ranges is not None else [(0, n)]):
        begin, count = int(begin), int(count)
        if count > 1:
            perm[begin:begin + count] = begin + _range_order(means[begin:begin + count].contiguous())
    return perm


def _range_order(m: torch.Tensor) -> torch.Tensor:
    count = m.shape[0]
    finite = torch.isfinite(m).all(dim=1)
    mf = m[finite] if not bool(finite.all()) else m
    lo = mf.min(dim=0).values.tolist() if mf.numel() else [0.0, 0.0, 0.0]
    hi = mf.max(dim=0).values.tolist() if mf.numel() else [0.0, 0.0, 0.0]
    codes = torch.empty(count, dtype=torch.int64, device=m.device)
    _lib.gs_spatial_codes(m, lo + hi, codes)
    # the codes are unsigned: flip the top bit so that signed order is their order
    key = codes ^ torch.iinfo(torch.int64).min
    return torch.argsort(key, stable=True)


def reorder(g: Gaussians, perm: torch.Tensor) -> Gaussians:
    """The Gaussians with every parameter tensor gathered by perm."""
    f = lambda t: t.index_select(0, perm).contiguous()
    return Gaussians(f(g.means), f(g.log_scales), f(g.quats), f(g.opacity_logits), f(g.sh))
