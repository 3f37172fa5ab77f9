"""Checkpoint and resume of a joint pose + 3DGS training run (off the hot
path).

A checkpoint holds everything a step of the training loop reads and updates:
the Gaussian parameters (means, log-scales, quaternions, opacity logits, SH
coefficients), the per-view pose residuals (6D rotation and translation,
Section 3.4), the optimiser state (Adam moments per parameter group and the
step count of the Eq. 1 update), and the random-number state the loop draws
its exploration noise and minibatches from. It is written atomically (to a
temporary file, then renamed), so an interrupted save leaves the previous
checkpoint intact.
"""
from __future__ import annotations

import os

import torch

from ._lib import Gaussians

GAUSSIAN_FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def save(path, gaussians: Gaussians, step: int, pose_residuals=None, optimizer_state=None, generators=None,
         extra=None):
    """Write a checkpoint. pose_residuals: dict name -> tensor (e.g. {"dr":
    [V,6], "dt": [V,3]}); optimizer_state: dict name -> (exp_avg,
    exp_avg_sq); generators: dict name -> torch.Generator (their states are
    saved); extra: any picklable metadata."""
    state = {
        "version": 1,
        "step": int(step),
        "gaussians": {k: getattr(gaussians, k).detach().cpu() for k in GAUSSIAN_FIELDS},
        "pose_residuals": {k: v.detach().cpu() for k, v in (pose_residuals or {}).items()},
        "optimizer": {k: (m.detach().cpu(), v.detach().cpu()) for k, (m, v) in (optimizer_state or {}).items()},
        "generators": {k: g.get_state() for k, g in (generators or {}).items()},
        "extra": extra,
    }
    path = os.fspath(path)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    torch.save(state, tmp)
    os.replace(tmp, path)


def load(path, device="cpu", generators=None):
    """Read a checkpoint; tensors are moved to device. Returns a dict with
    "step", "gaussians" (a Gaussians on device, or the raw tensors when device
    is the CPU), "pose_residuals", "optimizer" and "extra"; the states of the
    given generators (dict name -> torch.Generator) are restored in place."""
    state = torch.load(os.fspath(path), map_location="cpu", weights_only=False)
    if state.get("version") != 1:
        raise ValueError(f"unknown checkpoint version {state.get('version')!r}")
    dev = torch.device(device)
    gt = {k: v.to(dev).contiguous() for k, v in state["gaussians"].items()}
    out = {
        "step": state["step"],
        "gaussians": Gaussians(*(gt[k] for k in GAUSSIAN_FIELDS)) if dev.type == "cuda" else gt,
        "pose_residuals": {k: v.to(dev) for k, v in state["pose_residuals"].items()},
        "optimizer": {k: (m.to(dev), v.to(dev)) for k, (m, v) in state["optimizer"].items()},
        "extra": state["extra"],
    }
    for k, g in (generators or {}).items():
        g.set_state(state["generators"][k])
    return out
