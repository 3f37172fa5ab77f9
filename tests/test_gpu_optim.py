"""Parity of the fused SGLD/Adam update (Eq. 1) with the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle.optim import adam_sgld_step
from paper_2509_25191_gb300 import _lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 37, 50_000])
def test_sgld_adam_matches_oracle(n):
    rng = np.random.default_rng(n)
    shapes = [(n, 3), (n, 3), (n, 4), (n,), (n, 16, 3)]
    lrs = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]
    p32 = [rng.standard_normal(s).astype(np.float32) for s in shapes]
    ref = [dict(param=p.astype(np.float64), m=np.zeros(p.shape), v=np.zeros(p.shape), lr=lr, grad=None)
           for p, lr in zip(p32, lrs)]
    dev = [tuple(torch.as_tensor(x).cuda() for x in (p, np.zeros_like(p), np.zeros_like(p), np.zeros_like(p)))
           for p in p32]
    for step in (1, 2, 3):
        grads = [rng.standard_normal(s).astype(np.float32) for s in shapes]
        noise = rng.standard_normal((n, 3)).astype(np.float32)
        for r, g in zip(ref, grads):
            r["grad"] = g.astype(np.float64)
        adam_sgld_step(ref, step, noise=noise.astype(np.float64), noise_scale=0.01, noise_group=0)
        groups = []
        for (p, _, m, v), g, lr in zip(dev, grads, lrs):
            groups.append((p, torch.as_tensor(g).cuda(), m, v, lr))
        _lib.gs_sgld_adam_step(groups, step, noise=torch.as_tensor(noise).cuda(), noise_scale=0.01, noise_group=0)
        torch.cuda.synchronize()
        for (p, _, m, v), r in zip(dev, ref):
            assert np.allclose(p.cpu().numpy(), r["param"], rtol=1e-6, atol=1e-6 * r["lr"] + 1e-7)
            assert np.allclose(m.cpu().numpy(), r["m"], rtol=1e-5, atol=1e-7)
            assert np.allclose(v.cpu().numpy(), r["v"], rtol=1e-5, atol=1e-9)


def test_sgld_adam_rejects_bad_arguments():
    p = torch.zeros(4, device="cuda")
    with pytest.raises(_lib.GsError):
        _lib.gs_sgld_adam_step([(p, p, p, p, 1e-3)], 0)
    with pytest.raises(_lib.GsError):
        _lib.gs_sgld_adam_step([(p, p, p, p, 1e-3)], 1, noise=p, noise_group=3)
