"""gs_project_bwd_noalloc, the entry point for callers that cannot allocate
device memory (memory planners, plugin hosts, servers that forbid cudaMalloc
after start-up): called through the C ABI, it must give the same gradients as
gs_project_bwd + gs_pose_grad with caller-owned scratch, on consecutive calls
that share its static scratch array. Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2509_25191_gb300 import _lib, synth
from paper_2509_25191_gb300.autograd import Rasterizer
from tests.gpu_util import check_grad

pytestmark = pytest.mark.gpu


def _case():
    sc, vw = synth.orbit_views(3, 12000, 3, 160, 96, 1000.0 * 160 / 979.0)
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    rast = Rasterizer()
    image, proj = rast.forward(g, views)
    torch.cuda.synchronize()
    rast.check_status()
    return g, views, rast, image, proj


def test_noalloc_declared_and_exported():
    lib = _lib.load()
    assert hasattr(lib, "gs_project_bwd_noalloc")
    lib.gs_error_string.restype = ctypes.c_char_p
    assert b"allocation-free" in lib.gs_error_string(_lib.GS_ERR_TOO_LARGE)


def test_noalloc_matches_scratch_entry_point_on_consecutive_calls():
    g, views, rast, image, proj = _case()
    cfg = rast.cfg
    ref_grads = _lib.Grads(g.n, g.sh_degree, views.num_slots(), views.n)
    na_grads = _lib.Grads(g.n, g.sh_degree, views.num_slots(), views.n)
    for call, seed in enumerate((11, 12)):
        up = torch.as_tensor(np.random.default_rng(seed).standard_normal(views.num_image_floats())
                             .astype(np.float32)).cuda()
        # the 2D gradients both paths start from
        _lib.gs_rasterize_bwd(views, cfg, proj, rast.bins, image, up, ref_grads.grad2d)
        na_grads.grad2d.copy_(ref_grads.grad2d)
        # existing path: caller-owned pose partials
        _lib.gs_project_bwd(g, views, cfg, proj, ref_grads)
        ref_vm = torch.empty(views.n, 12, device="cuda")
        ref_tw = torch.empty(views.n, 6, device="cuda")
        _lib.gs_pose_grad(views, ref_grads.pose_partials, ref_grads.n_blocks, ref_vm, ref_tw)
        # allocation-free path
        vm = torch.full((views.n, 12), float("nan"), device="cuda")
        tw = torch.full((views.n, 6), float("nan"), device="cuda")
        _lib.gs_project_bwd_noalloc(g, views, cfg, proj, na_grads, vm, tw)
        torch.cuda.synchronize()
        for name in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
            check_grad(getattr(na_grads, name).cpu().numpy(), getattr(ref_grads, name).cpu().numpy(),
                       f"call {call}: {name}")
        check_grad(vm.cpu().numpy(), ref_vm.cpu().numpy(), f"call {call}: dL/d(R,t)")
        check_grad(tw.cpu().numpy(), ref_tw.cpu().numpy(), f"call {call}: twist")
