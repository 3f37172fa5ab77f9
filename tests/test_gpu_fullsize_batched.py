"""Parity at the full sizes of the batched workloads, through the captured
training step (GraphStep) at the autotuner's tile and batch, where the oracle can
afford it:

* 16 views 979x546 on the radius-5 orbit of one 500K-Gaussian clustered SH3
  scene (the batched-versus-plain workload);
* one minibatch of the dense joint pose step: 8 of the 300 jittered
  hemisphere views, 1600x1066, of the 6M-Gaussian SH3 scene (hundreds of
  millions of tile instances, tiles far above the on-chip sort size).

The image is checked on a random sample of pixels per view. For the
gradients the step's own L1 loss is used with a target equal to the rendered
image except on sampled pixels, where it differs by +-0.5: the loss gradient
the captured step computes is then sign/count on those pixels and exactly
zero elsewhere, and the oracle's backward with that upstream gradient checks
every Gaussian parameter and every view's pose."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_25191_gb300 import _lib, synth
from paper_2509_25191_gb300.step import GraphStep
from paper_2509_25191_gb300.tune import autotune
from tests.gpu_util import check_grad, image_errors, split

pytestmark = pytest.mark.gpu

SORT_ON_CHIP = 4096   # keys one block sorts on chip; larger tiles take the partition pass


def _masks(vw, per_view, seed):
    rng = np.random.default_rng(seed)
    masks = []
    for v in range(vw.n):
        W, H = int(vw.width[v]), int(vw.height[v])
        m = np.zeros((H, W), bool)
        m.reshape(-1)[rng.choice(W * H, per_view, replace=False)] = True
        m[-3:, :] = True          # the ragged last row and column of tiles
        m[:, -3:] = True
        masks.append(m)
    return masks


def _run(sc, vw, per_view, seed):
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    target = torch.zeros(views.num_image_floats(), device="cuda")
    choice, _ = autotune(g, views, target, reps=3)
    step = GraphStep(g, views, target, tile=choice.tile, batch=choice.batch)
    step.replay()
    assert step.check() is False
    torch.cuda.synchronize()
    masks = _masks(vw, per_view, seed)
    ref = O.forward(sc, vw, masks=masks)
    imgs = split(step.image, vw)
    err, flagged = image_errors(imgs, ref, masks)
    n_masked = sum(int(m.sum()) for m in masks)
    assert flagged <= 0.05 * n_masked   # pixels at a threshold within the FP32 margin (at most a few %)
    assert err <= 1e-4, err
    # sparse upstream through the step's own L1 loss
    rng = np.random.default_rng(seed + 1)
    count = views.num_image_floats()
    ups, tgt = [], []
    for v in range(vw.n):
        W, H = int(vw.width[v]), int(vw.height[v])
        pick = masks[v] & ((ref[v]["flags"] & O.GRAD_FLAGS) == 0) & (rng.random((H, W)) < 0.5)
        s = np.zeros((3, H, W), np.float32)
        s[:, pick] = rng.choice([-1.0, 1.0], size=(3, int(pick.sum())))
        ups.append(s.astype(np.float64) / count)
        tgt.append((imgs[v] - 0.5 * s).reshape(-1))
    step.target.copy_(torch.as_tensor(np.concatenate(tgt)))
    step.replay()
    assert step.check() is False
    torch.cuda.synchronize()
    n_up = sum(int((u != 0).any(0).sum()) for u in ups)
    loss_want = 0.5 * sum(int((u != 0).sum()) for u in ups) / count
    assert abs(float(step.loss[0]) - loss_want) <= 1e-5 * loss_want
    rg, dRt, tw, _ = O.backward(sc, vw, ref, ups)
    for name in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        check_grad(getattr(step.grads, name).cpu().numpy(), rg[name], name)
    check_grad(step.dviewmat.cpu().numpy(), dRt, "dL/d(R,t)")
    check_grad(step.dtwist.cpu().numpy(), tw, "twist")
    return step, choice, n_up


def test_orbit_16_views_500k_full_size():
    sc, vw = synth.orbit_views(0, 500_000, 16, 979, 546)
    step, choice, n_up = _run(sc, vw, per_view=1500, seed=31)
    assert n_up > 5000
    assert int(step.bins.counters[0].item()) > 1_000_000


def test_dense_minibatch_8_views_6m_full_size():
    sc, true_v, noisy_v = synth.dense_hemisphere(0)
    vw = noisy_v.select(synth.minibatch(0, noisy_v.n, 8))
    step, choice, n_up = _run(sc, vw, per_view=1000, seed=41)
    assert n_up > 2000
    assert int(step.bins.counters[0].item()) > 50_000_000
    assert int(step.bins.counters[6].item()) > 4 * SORT_ON_CHIP   # the largest tile takes the partition pass
