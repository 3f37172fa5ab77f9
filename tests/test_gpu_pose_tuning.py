"""Test-time pose tuning (Gaussians frozen, backward to the pose only)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_25191_gb300 import _lib, pose, synth
from paper_2509_25191_gb300.autograd import Rasterizer
from paper_2509_25191_gb300.step import GraphStep
from tests.gpu_util import check_grad, oracle_forward, upstream

pytestmark = pytest.mark.gpu


def test_pose_only_gradient_matches_oracle():
    sc, vw = synth.orbit_views(2, 20000, 3, 160, 96, 160.0)
    ref = oracle_forward(sc, vw)
    ups = upstream(vw, ref, seed=3)
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    rast = Rasterizer()
    image, proj = rast.forward(g, views)
    up = torch.as_tensor(np.concatenate([u.reshape(-1) for u in ups])).cuda()
    _, dvm, dtw = rast.backward(g, views, proj, image, up, want_gaussian_grads=False)
    torch.cuda.synchronize()
    _, dRt, tw, _ = O.backward(sc, vw, ref, [u.astype(np.float64) for u in ups])
    check_grad(dvm.cpu().numpy(), dRt, "pose-only dL/d(R,t)")
    check_grad(dtw.cpu().numpy(), tw, "pose-only twist")


def test_pose_only_tuning_recovers_a_jittered_pose():
    """Frozen Gaussians, target rendered from the true pose; Adam on the 6D
    and translation residuals of a pose perturbed by 1 degree / 1 %, with the
    pose-only captured step (L1 loss), must bring the pose back."""
    sc, vw = synth.orbit_views(4, 60000, 1, 240, 160, 240.0)
    g = _lib.Gaussians.from_scene(sc)
    true_vm = torch.as_tensor(vw.viewmats).cuda()
    noisy = torch.as_tensor(synth.jitter_viewmats(vw.viewmats, seed=9).astype(np.float32)).cuda()
    intr = torch.as_tensor(vw.intrinsics).cuda()
    target, _ = Rasterizer().forward(g, _lib.Views(true_vm, intr, vw.width, vw.height, vw.gauss_begin,
                                                   vw.gauss_count))
    vm_static = noisy.clone()
    views = _lib.Views(vm_static, intr, vw.width, vw.height, vw.gauss_begin, vw.gauss_count)
    step = GraphStep(g, views, target.clone(), want_gaussian_grads=False)
    dr = pose.identity_6d(1, device="cuda").requires_grad_(True)
    dt = torch.zeros(1, 3, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([dr, dt], lr=2e-3)

    def pose_error(vm):
        R, Rt = vm[0, :9].reshape(3, 3), true_vm[0, :9].reshape(3, 3)
        ang = torch.arccos(torch.clamp((torch.trace(R @ Rt.T) - 1) / 2, -1, 1)) * 180 / np.pi
        return float(ang), float((vm[0, 9:] - true_vm[0, 9:]).norm())

    a0, t0 = pose_error(noisy)
    losses = []
    for it in range(150):
        vm = pose.apply_residual(noisy, dr, dt)
        with torch.no_grad():
            vm_static.copy_(vm)
        step.replay()
        opt.zero_grad()
        vm.backward(step.dviewmat)
        opt.step()
        losses.append(float(step.loss.item()))
    torch.cuda.synchronize()
    assert not step.check()
    a1, t1 = pose_error(pose.apply_residual(noisy, dr, dt).detach())
    assert losses[-1] < 0.5 * losses[0]
    assert a1 < 0.35 * a0 and t1 < 0.5 * t0, (a0, a1, t0, t1)
