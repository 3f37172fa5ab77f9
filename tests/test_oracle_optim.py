"""Pins of the FP64 SGLD/Adam oracle (Eq. 1)."""
import numpy as np
import torch

from oracle.optim import adam_sgld_step


def _groups(seed=0):
    rng = np.random.default_rng(seed)
    shapes, lrs = [(50, 3), (50, 3), (50, 4), (50,), (50, 16, 3)], [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]
    return [dict(param=rng.standard_normal(s), grad=None, m=np.zeros(s), v=np.zeros(s), lr=lr)
            for s, lr in zip(shapes, lrs)], rng


def test_matches_torch_adam_over_several_steps():
    groups, rng = _groups()
    tparams = [torch.tensor(g["param"].copy(), requires_grad=True) for g in groups]
    opt = torch.optim.Adam([dict(params=[t], lr=g["lr"]) for t, g in zip(tparams, groups)], betas=(0.9, 0.999),
                           eps=1e-15)
    for step in range(1, 6):
        grads = [rng.standard_normal(g["param"].shape) for g in groups]
        for g, gr in zip(groups, grads):
            g["grad"] = gr
        adam_sgld_step(groups, step)
        for t, gr in zip(tparams, grads):
            t.grad = torch.tensor(gr)
        opt.step()
        for g, t in zip(groups, tparams):
            assert np.allclose(g["param"], t.detach().numpy(), rtol=1e-12, atol=1e-12)


def test_first_step_closed_form_and_noise():
    groups, rng = _groups(1)
    p0 = [g["param"].copy() for g in groups]
    for g in groups:
        g["grad"] = rng.standard_normal(g["param"].shape)
    noise = rng.standard_normal((50, 3))
    adam_sgld_step(groups, 1, eps=1e-15, noise=noise, noise_scale=0.02, noise_group=0)
    # step 1: m_hat = g, v_hat = g^2, so the step is lr * sign(g)
    for k, (g, p) in enumerate(zip(groups, p0)):
        expect = p - g["lr"] * np.sign(g["grad"]) + (0.02 * noise if k == 0 else 0.0)
        assert np.allclose(g["param"], expect, rtol=0, atol=1e-12)
