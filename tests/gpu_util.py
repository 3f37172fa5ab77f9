"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded inputs and compare."""
import numpy as np
import torch

from oracle import oracle as O
from paper_2509_25191_gb300 import _lib
from paper_2509_25191_gb300.autograd import Rasterizer


def gpu_forward(scene, views, tile=(16, 16), bg=(0.0, 0.0, 0.0), rast=None):
    rast = rast or Rasterizer(tile=tile, bg=bg)
    g = _lib.Gaussians.from_scene(scene)
    vw = _lib.Views.from_synth(views)
    image, proj = rast.forward(g, vw)
    torch.cuda.synchronize()
    rast.check_status()
    return rast, g, vw, image, proj


def split(image, views):
    out, off = [], 0
    img = image.detach().cpu().numpy() if torch.is_tensor(image) else image
    for v in range(views.n):
        W, H = int(views.width[v]), int(views.height[v])
        out.append(img[off:off + 3 * W * H].reshape(3, H, W))
        off += 3 * W * H
    return out


def oracle_forward(scene, views, tile=(16, 16), bg=(0.0, 0.0, 0.0), masks=None):
    return O.forward(scene, views, tile[0], tile[1], O.Params(bg=bg), masks)


def image_errors(gpu_imgs, ref, masks=None):
    """Max abs error over unflagged (and, if given, masked-in) pixels; number
    of flagged pixels."""
    worst, flagged = 0.0, 0
    for v, r in enumerate(ref):
        ok = (r["flags"] & O.IMAGE_FLAGS) == 0
        if masks is not None:
            ok &= masks[v]
            flagged += int(((r["flags"] & O.IMAGE_FLAGS) != 0)[masks[v]].sum())
        else:
            flagged += int((~ok).sum())
        if ok.any():
            worst = max(worst, float(np.abs(gpu_imgs[v] - r["image"])[:, ok].max()))
    return worst, flagged


def upstream(views, ref, seed=1, masks=None):
    """Random dL/dimage per view (float32 values), zero at pixels flagged for
    gradients and outside masks."""
    rng = np.random.default_rng(seed)
    ups = []
    for v in range(views.n):
        W, H = int(views.width[v]), int(views.height[v])
        u = rng.standard_normal((3, H, W)).astype(np.float32)
        u[:, (ref[v]["flags"] & O.GRAD_FLAGS) != 0] = 0.0
        if masks is not None:
            u[:, ~masks[v]] = 0.0
        ups.append(u)
    return ups


def conic_to_cov_grads(g2d, conic):
    """Oracle 2D gradients w.r.t. (x, y, A, B, C, o, r, g, b) with the conic
    (A, B, C) -> the same w.r.t. the covariance (a, b, c) it inverts:
    G_cov = -Q G_Q Q with G_Q = [[gA, gB/2], [gB/2, gC]] (FP64, exact map)."""
    out = np.array(g2d, np.float64, copy=True)
    A, B, C = conic[:, 0], conic[:, 1], conic[:, 2]
    Q = np.stack([np.stack([A, B], -1), np.stack([B, C], -1)], -2)
    G = np.stack([np.stack([g2d[:, 2], 0.5 * g2d[:, 3]], -1), np.stack([0.5 * g2d[:, 3], g2d[:, 4]], -1)], -2)
    Gc = -Q @ G @ Q
    out[:, 2], out[:, 3], out[:, 4] = Gc[:, 0, 0], 2 * Gc[:, 0, 1], Gc[:, 1, 1]
    return out


def check_grad(g, ref, what, rel_norm=1e-3, rel_elem=1e-3, abs_frac=1e-5):
    """Gradient tolerance: ||g - g*|| <= 1e-3 ||g*|| and elementwise
    |g - g*| <= 1e-3 |g*| + 1e-5 max|g*|."""
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nr = np.linalg.norm(ref)
    if nr == 0:
        assert np.abs(g).max() == 0, what
        return 0.0
    rel = np.linalg.norm(g - ref) / nr
    assert rel <= rel_norm, f"{what}: relative norm error {rel:.3e}"
    bound = rel_elem * np.abs(ref) + abs_frac * np.abs(ref).max()
    bad = np.abs(g - ref) > bound
    if bad.any():
        w = int(np.argmax(np.abs(g - ref) - bound))
        raise AssertionError(f"{what}: {bad.sum()} of {g.size} elements out of bound; worst at {w}: got {g[w]:.6e} "
                             f"want {ref[w]:.6e} bound {bound[w]:.3e} max|g*| {np.abs(ref).max():.3e} "
                             f"norm rel {rel:.2e}")
    return rel
