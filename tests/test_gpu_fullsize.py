"""Parity at the benchmark's full size (1,000,000 clustered SH3 Gaussians, one
1237x822 view, 32x16 tiles: the configuration bench.py times, its
autotuner's choice on this workload), checked where
the oracle can afford it: a random sample of pixels for the image, and an
upstream gradient that is non-zero only on sampled pixels for the backward
(every Gaussian parameter and the pose still get checked)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_25191_gb300 import _lib, synth
from paper_2509_25191_gb300.autograd import Rasterizer
from tests.gpu_util import check_grad, split

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    sc, vw = synth.single_view_1m()
    rast = Rasterizer(tile=(32, 16))
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    image, proj = rast.forward(g, views)
    torch.cuda.synchronize()
    rast.check_status()
    W, H = int(vw.width[0]), int(vw.height[0])
    rng = np.random.default_rng(2024)
    mask = np.zeros((H, W), bool)
    mask.reshape(-1)[rng.choice(W * H, 20000, replace=False)] = True
    mask[:16, :] = True            # one full row of tiles, and the ragged last row and column
    mask[-6:, :] = True
    mask[:, -5:] = True
    ref = O.forward(sc, vw, masks=[mask])[0]
    return sc, vw, rast, g, views, image, proj, mask, ref


def test_full_size_image_on_sampled_pixels(full):
    sc, vw, rast, g, views, image, proj, mask, ref = full
    img = split(image, vw)[0]
    ok = mask & ((ref["flags"] & O.IMAGE_FLAGS) == 0)
    assert ok.sum() > 0.95 * mask.sum()
    err = np.abs(img - ref["image"])[:, ok].max()
    assert err <= 1e-4, err
    assert rast.last_instances > 1_000_000


def test_full_size_gradients_with_sparse_upstream(full):
    sc, vw, rast, g, views, image, proj, mask, ref = full
    W, H = int(vw.width[0]), int(vw.height[0])
    rng = np.random.default_rng(7)
    up = np.zeros((3, H, W), np.float32)
    pick = mask & ((ref["flags"] & O.GRAD_FLAGS) == 0) & (rng.random((H, W)) < 0.25)
    up[:, pick] = rng.standard_normal((3, int(pick.sum()))).astype(np.float32)
    grads, dvm, dtw = rast.backward(g, views, proj, image, torch.as_tensor(up.reshape(-1)).cuda())
    torch.cuda.synchronize()
    rg, dRt, tw, _ = O.backward(sc, vw, [ref], [up.astype(np.float64)])
    touched = np.abs(rg["means"]).sum(1) > 0
    assert touched.sum() > 1000
    for name in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        check_grad(getattr(grads, name).cpu().numpy(), rg[name], name)
    check_grad(dvm.cpu().numpy(), dRt, "dL/d(R,t)")
    check_grad(dtw.cpu().numpy(), tw, "twist")
