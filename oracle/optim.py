"""FP64 oracle of the SGLD update with an Adam direction (paper Eq. 1).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline); shares no code
with the CUDA library.

Eq. 1 updates the Gaussians by a learning-rate-scaled gradient step plus
exploration noise: G <- G - lr * step(grad) + lambda_noise * eps. The step
follows the attribute schedule of the cited MCMC-3DGS training, i.e. Adam:
    m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
    p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps_adam),
and the exploration noise (drawn by the caller, so both sides see the same
numbers) is added to one parameter group, the Gaussian means:
    p <- p + noise_scale * eps.
Pinned in tests against torch.optim.Adam (an independent implementation)
and against the first-step closed form m_hat = g, v_hat = g^2.
"""
import numpy as np


def adam_sgld_step(groups, step, beta1=0.9, beta2=0.999, eps=1e-15, noise=None, noise_scale=0.0,
                   noise_group=0):
    """groups: list of dicts with param, grad, m, v (arrays, updated in place
    in float64) and lr. step: 1-based Adam step count."""
    bc1 = 1.0 - beta1 ** step
    bc2 = 1.0 - beta2 ** step
    for k, gr in enumerate(groups):
        p, g, m, v = gr["param"], gr["grad"], gr["m"], gr["v"]
        m *= beta1
        m += (1.0 - beta1) * g
        v *= beta2
        v += (1.0 - beta2) * g * g
        p -= gr["lr"] * (m / bc1) / (np.sqrt(v / bc2) + eps)
        if noise is not None and k == noise_group:
            p += noise_scale * noise.reshape(p.shape)
    return groups
