"""Per-view residual pose (Section 3.4): translation residual dt in R^3 and
rotation residual dr in R^6, the 6D rotation representation turned into a
rotation matrix by Gram-Schmidt (columns b1, b2, b3 = b1 x b2), applied as
R' = dR R, t' = t + dt. Plain torch ops on V small matrices; the
rasterizer's dL/d(R', t') flows back through them by autograd.
"""
import torch


def rotation_6d(dr):
    """[V,6] -> [V,3,3]: a1 = dr[:, :3], a2 = dr[:, 3:];
    b1 = a1/|a1|, b2 = normalise(a2 - (b1.a2) b1), b3 = b1 x b2 (columns)."""
    a1, a2 = dr[:, :3], dr[:, 3:]
    b1 = a1 / a1.norm(dim=-1, keepdim=True)
    b2 = a2 - (b1 * a2).sum(-1, keepdim=True) * b1
    b2 = b2 / b2.norm(dim=-1, keepdim=True)
    b3 = torch.cross(b1, b2, dim=-1)
    return torch.stack([b1, b2, b3], dim=-1)


def identity_6d(n, device=None, dtype=torch.float32):
    return torch.tensor([1.0, 0.0, 0.0, 0.0, 1.0, 0.0], device=device, dtype=dtype).repeat(n, 1)


def apply_residual(viewmats, dr, dt):
    """viewmats [V,12] (R row-major, t) -> refined [V,12]."""
    R = viewmats[:, :9].reshape(-1, 3, 3)
    t = viewmats[:, 9:]
    Rn = rotation_6d(dr) @ R
    return torch.cat([Rn.reshape(-1, 9), t + dt], dim=1)


def pose_lr(step, total_steps=30000, lr0=1e-4, factor=0.1):
    """Learning rate of the pose residuals at training step ``step``
    (Section 4.1, implementation details: initialised at 1e-4 and decayed
    exponentially by a factor of 0.1 over the training run, whose length
    follows the MCMC-3DGS schedule, 30,000 iterations):
    lr0 * factor ** (step / total_steps), held at lr0 * factor afterwards."""
    if total_steps <= 0:
        raise ValueError("total_steps must be positive")
    return lr0 * factor ** (min(max(step, 0), total_steps) / total_steps)
