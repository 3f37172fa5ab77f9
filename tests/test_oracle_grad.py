"""Pins of the oracle's analytic backward: FP64 central finite differences of
the oracle's own forward, and an independent torch autograd restatement."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_25191_gb300 import synth
from paper_2509_25191_gb300.synth import Scene
from tests import torch_ref

W, H, TILE = 24, 20, 32   # one tile: no tile rectangle can change under perturbation


def _grad_scene(seed=0, n=6, deg=3):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.3, 0.3, n), rng.uniform(2.0, 4.0, n)], 1)
    ls = rng.normal(-2.6, 0.3, (n, 3))
    q = rng.standard_normal((n, 4))
    lg = rng.normal(0.0, 1.0, n)
    K = (deg + 1) ** 2
    sh = np.zeros((n, K, 3))
    sh[:, 0] = rng.uniform(-1.5, 1.5, (n, 3))
    sh[:, 1:] = rng.normal(0, 0.3, (n, K - 1, 3))
    # one Gaussian outside the tangent clamp whose footprint reaches the image
    means[-1] = [0.75 * 3.0, 0.0, 3.0]
    ls[-1] = math.log(0.35)
    sc = Scene(means, ls, q, lg, sh, deg)          # float64 arrays: FD runs in FP64
    cam = synth.look_at((0.15, -0.1, -0.2), target=(0.0, 0.0, 3.0))
    vw = synth.Views(cam.reshape(1, 12).astype(np.float64), np.array([[30.0, 32.0, 12.2, 9.7]]),
                     np.array([W], np.int32), np.array([H], np.int32), np.array([0]), np.array([n]))
    return sc, vw


def _loss(sc, vw, wts, prm):
    img = O.forward(sc, vw, TILE, TILE, prm)[0]["image"]
    return float((img * wts).sum())


def _weights(sc, vw, prm, seed=1):
    f = O.forward(sc, vw, TILE, TILE, prm)
    wts = np.random.default_rng(seed).standard_normal((3, H, W))
    wts[:, (f[0]["flags"] & O.GRAD_FLAGS) != 0] = 0.0
    return f, wts


def _check(fd, an, what):
    fd, an = np.asarray(fd), np.asarray(an)
    scale = np.abs(an).max() + 1e-30
    err = np.abs(fd - an)
    assert (err <= 1e-6 * scale + 1e-5 * np.abs(an)).all(), (what, err.max(), scale)


@pytest.mark.parametrize("seed,bg", [(0, (0.0, 0.0, 0.0)), (3, (0.3, 0.6, 0.1))])
def test_oracle_gradients_match_central_differences(seed, bg):
    sc, vw = _grad_scene(seed)
    prm = O.Params(bg=bg)
    f, wts = _weights(sc, vw, prm)
    assert f[0]["n_contrib"].max() >= 3
    grads, dRt, tw, _ = O.backward(sc, vw, f, [wts], TILE, TILE, prm)
    h = 1e-6
    for name in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        arr = getattr(sc, name)
        fd = np.zeros_like(arr)
        flat = arr.reshape(-1)
        for j in range(flat.size):
            old = flat[j]
            flat[j] = old + h
            lp = _loss(sc, vw, wts, prm)
            flat[j] = old - h
            lm = _loss(sc, vw, wts, prm)
            flat[j] = old
            fd.reshape(-1)[j] = (lp - lm) / (2 * h)
        _check(fd, grads[name], name)
    # pose entries (R treated as 9 free entries, then t)
    fd = np.zeros(12)
    for j in range(12):
        old = vw.viewmats[0, j]
        vw.viewmats[0, j] = old + h
        lp = _loss(sc, vw, wts, prm)
        vw.viewmats[0, j] = old - h
        lm = _loss(sc, vw, wts, prm)
        vw.viewmats[0, j] = old
        fd[j] = (lp - lm) / (2 * h)
    _check(fd, dRt[0], "R,t")
    # left twist (rho, phi): T <- exp(xi^) T
    base = vw.viewmats[0].copy()
    R0, t0 = base[:9].reshape(3, 3), base[9:]
    fdt = np.zeros(6)
    for k in range(6):
        vals = []
        for sgn in (1, -1):
            if k < 3:
                Rn, tn = R0, t0 + sgn * h * np.eye(3)[k]
            else:
                Rot = synth._axis_angle(np.eye(3)[k - 3], sgn * h)
                Rn, tn = Rot @ R0, Rot @ t0
            vw.viewmats[0] = np.concatenate([Rn.reshape(-1), tn])
            vals.append(_loss(sc, vw, wts, prm))
        vw.viewmats[0] = base
        fdt[k] = (vals[0] - vals[1]) / (2 * h)
    _check(fdt, tw[0], "twist")


def test_oracle_gradients_match_torch_autograd():
    sc, vw = _grad_scene(5, n=7)
    prm = O.Params(bg=(0.2, 0.1, 0.4))
    f, wts = _weights(sc, vw, prm, seed=4)
    grads, dRt, _, _ = O.backward(sc, vw, f, [wts], TILE, TILE, prm)
    t64 = lambda a: torch.tensor(np.asarray(a, np.float64), requires_grad=True)
    p = {k: t64(getattr(sc, k)) for k in ["means", "log_scales", "quats", "opacity_logits", "sh"]}
    R = t64(vw.viewmats[0, :9].reshape(3, 3))
    t = t64(vw.viewmats[0, 9:])
    fx, fy, cx, cy = [float(v) for v in vw.intrinsics[0]]
    img = torch_ref.render(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"], R, t,
                           fx, fy, cx, cy, W, H, bg=prm.bg)
    assert np.abs(img.detach().numpy() - f[0]["image"]).max() < 1e-12
    (img * torch.tensor(wts)).sum().backward()
    for k in p:
        _check(p[k].grad.numpy(), grads[k], k)
    _check(R.grad.numpy().reshape(-1), dRt[0, :9], "R")
    _check(t.grad.numpy(), dRt[0, 9:], "t")
