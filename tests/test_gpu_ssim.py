"""GPU parity of the fused L1 + D-SSIM loss (Section 3.1) against the FP64
oracle, through the C ABI: ragged multi-view images (tiles cut by the image
border), the full 1237x822 size, identical images."""
import numpy as np
import pytest
import torch

from oracle import ssim as OS
from paper_2509_25191_gb300 import _lib
from tests.gpu_util import check_grad

pytestmark = pytest.mark.gpu


def _images(shapes, seed):
    """Smooth fields with edges and noise, and a perturbed copy."""
    rng = np.random.default_rng(seed)
    ims, tgs = [], []
    for (H, W) in shapes:
        yy, xx = np.mgrid[0:H, 0:W] / max(H, W)
        base = np.stack([0.5 + 0.4 * np.sin(6 * xx + k) * np.cos(4 * yy - k) for k in range(3)])
        base[:, :, W // 2:] += 0.2
        tg = np.clip(base + 0.05 * rng.standard_normal(base.shape), 0, 1)
        im = np.clip(tg + 0.1 * rng.standard_normal(base.shape), 0, 1)
        ims.append(im.astype(np.float32))
        tgs.append(tg.astype(np.float32))
    return ims, tgs


def _gpu(ims, tgs, lam=0.2):
    W = [im.shape[2] for im in ims]
    H = [im.shape[1] for im in ims]
    views = _lib.Views(None, None, W, H, [0] * len(W), [0] * len(W))
    x = torch.as_tensor(np.concatenate([im.reshape(-1) for im in ims])).cuda()
    y = torch.as_tensor(np.concatenate([t.reshape(-1) for t in tgs])).cuda()
    loss = torch.full((3,), float("nan"), device="cuda")
    g = torch.full_like(x, float("nan"))
    _lib.gs_l1_dssim_loss(views, x, y, loss, g, lam)
    torch.cuda.synchronize()
    out, off = [], 0
    gh = g.cpu().numpy()
    for im in ims:
        out.append(gh[off:off + im.size].reshape(im.shape))
        off += im.size
    return loss.cpu().numpy(), out


def _check(ims, tgs, lam=0.2):
    loss, grads = _gpu(ims, tgs, lam)
    total, l1, dssim, ref = OS.l1_dssim(ims, tgs, lam)
    assert abs(loss[1] - l1) <= 1e-5 * max(l1, 1e-3), (loss, l1)
    assert abs(loss[2] - dssim) <= 2e-6 + 1e-5 * dssim, (loss, dssim)
    assert abs(loss[0] - total) <= 2e-6 + 1e-5 * total
    check_grad(np.concatenate([g.reshape(-1) for g in grads]), np.concatenate([r.reshape(-1) for r in ref]),
               "dL/dimage")


def test_ragged_multi_view_parity():
    _check(*_images([(70, 52), (33, 90), (1, 1), (32, 64)], 0))


def test_lambda_extremes():
    ims, tgs = _images([(40, 45)], 1)
    _check(ims, tgs, 0.0)
    _check(ims, tgs, 1.0)


def test_full_size_parity():
    _check(*_images([(822, 1237)], 2))


def test_identical_images():
    ims, _ = _images([(50, 61)], 3)
    loss, grads = _gpu(ims, [im.copy() for im in ims])
    assert loss[1] == 0 and abs(loss[2]) < 1e-6 and abs(loss[0]) < 1e-6
    # zero up to float32 cancellation in 2x G(b) + y G(c), far below the 1/n scale
    assert np.abs(grads[0]).max() < 1e-3 / ims[0].size
