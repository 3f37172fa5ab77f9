"""An independent FP64 restatement of the rasterizer in plain torch ops, used
only by the tests as a third opinion on the oracle's analytic gradients.

It is written from the mathematics with different building blocks than the
C oracle: the rotation comes from Hamilton products, the SH from the
associated-Legendre recurrence, the conic from ``torch.linalg.inv``, and the
gradient from autograd. Discrete decisions (culling, radius, gate, alpha
cutoff, early stop) are taken without gradient, as in the method. Meant for a
handful of Gaussians on a single-tile image.
"""
import math

import torch


def _hamilton(a, b):
    w1, x1, y1, z1 = a.unbind(-1)
    w2, x2, y2, z2 = b.unbind(-1)
    return torch.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                        w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], -1)


def rotation_from_quats(q):
    """[n,4] -> [n,3,3]: columns are q e_k q* (unit-normalised q)."""
    q = q / q.norm(dim=-1, keepdim=True)
    qc = q * torch.tensor([1.0, -1.0, -1.0, -1.0], dtype=q.dtype)
    cols = []
    for k in range(3):
        e = torch.zeros(q.shape[0], 4, dtype=q.dtype)
        e[:, k + 1] = 1.0
        cols.append(_hamilton(_hamilton(q, e), qc)[:, 1:])
    return torch.stack(cols, -1)


def sh_basis(deg, d):
    """[n,3] unit directions -> [n,(deg+1)^2], real SH with Condon-Shortley
    phase via Q_l^m with P_l^m = (1-z^2)^(m/2) Q_l^m."""
    x, y, z = d.unbind(-1)
    out = [None] * (deg + 1) ** 2
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for m in range(1, deg + 1):
        re.append(re[-1] * x - im[-1] * y)
        im.append(re[-2] * y + im[-1] * x)
    for m in range(deg + 1):
        dfact = 1.0
        for k in range(1, 2 * m, 2):
            dfact *= k
        Q = {m: torch.full_like(z, (-1) ** m * dfact)}
        if m + 1 <= deg:
            Q[m + 1] = z * (2 * m + 1) * Q[m]
        for l in range(m + 2, deg + 1):
            Q[l] = ((2 * l - 1) * z * Q[l - 1] - (l + m - 1) * Q[l - 2]) / (l - m)
        for l in range(m, deg + 1):
            K = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))
            if m == 0:
                out[l * l + l] = K * Q[l]
            else:
                out[l * l + l + m] = math.sqrt(2) * K * Q[l] * re[m]
                out[l * l + l - m] = math.sqrt(2) * K * Q[l] * im[m]
    return torch.stack(out, -1)


def render(means, log_scales, quats, logits, sh, R, t, fx, fy, cx, cy, W, H,
           near=0.2, dilation=0.3, alpha_min=1 / 255, alpha_max=0.99, t_min=1e-4, fov_clamp=1.3,
           bg=(0.0, 0.0, 0.0)):
    """Image [3,H,W] of one view; R [3,3], t [3] world->camera."""
    dt = torch.float64
    n = means.shape[0]
    deg = int(round(math.sqrt(sh.shape[1]))) - 1
    mc = means @ R.T + t
    x, y, z = mc.unbind(-1)
    Rq = rotation_from_quats(quats)
    S = torch.exp(log_scales)
    M = Rq * S[:, None, :]
    Sig = M @ M.transpose(1, 2)
    limx = fov_clamp * 0.5 * W / fx
    limy = fov_clamp * 0.5 * H / fy
    u = torch.clamp(x / z, -limx, limx)
    w = torch.clamp(y / z, -limy, limy)
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([fx / z, zero, -fx * u / z], -1),
                     torch.stack([zero, fy / z, -fy * w / z], -1)], -2)        # [n,2,3]
    Tm = J @ R
    cov = Tm @ Sig @ Tm.transpose(1, 2) + dilation * torch.eye(2, dtype=dt)
    conic = torch.linalg.inv(cov)
    px = fx * x / z + cx
    py = fy * y / z + cy
    o = torch.sigmoid(logits)
    C = -(R.T @ t)
    dirs = means - C
    d = dirs / dirs.norm(dim=-1, keepdim=True)
    Y = sh_basis(deg, d)
    rgb = torch.clamp((Y[:, :, None] * sh).sum(1) + 0.5, min=0.0)

    with torch.no_grad():
        a, b, c = cov[:, 0, 0], cov[:, 0, 1], cov[:, 1, 1]
        det = a * c - b * b
        mid = 0.5 * (a + c)
        lam = mid + torch.sqrt(torch.clamp(mid * mid - det, min=0.1))
        radius = torch.ceil(3 * torch.sqrt(lam))
        valid = (z > near) & (det > 0) & ~((px + radius < 0) | (px - radius > W) | (py + radius < 0) | (py - radius > H))
        zf = z.to(torch.float32)
        order = sorted(range(n), key=lambda i: (float(zf[i]), i))

    vv, uu = torch.meshgrid(torch.arange(H, dtype=dt), torch.arange(W, dtype=dt), indexing="ij")
    pcx, pcy = (uu + 0.5).reshape(-1), (vv + 0.5).reshape(-1)
    P = pcx.shape[0]
    T = torch.ones(P, dtype=dt)
    col = torch.zeros(P, 3, dtype=dt)
    stopped = torch.zeros(P, dtype=torch.bool)
    for g in order:
        if not bool(valid[g]):
            continue
        dx = pcx - px[g]
        dy = pcy - py[g]
        power = -0.5 * (conic[g, 0, 0] * dx * dx + conic[g, 1, 1] * dy * dy) - conic[g, 0, 1] * dx * dy
        oG = o[g] * torch.exp(power)
        alpha = torch.where(oG > alpha_max, torch.full_like(oG, alpha_max), oG)
        Tn = T * (1 - alpha)
        with torch.no_grad():
            ok = (dx.abs() <= radius[g]) & (dy.abs() <= radius[g]) & (power <= 0) & (alpha >= alpha_min) & ~stopped
            stop_now = ok & (Tn < t_min)
            stopped = stopped | stop_now
            use = ok & ~stop_now
        col = col + torch.where(use[:, None], rgb[g][None, :] * (alpha * T)[:, None], torch.zeros_like(col))
        T = torch.where(use, Tn, T)
    img = col + T[:, None] * torch.tensor(bg, dtype=dt)[None, :]
    return img.T.reshape(3, H, W)
