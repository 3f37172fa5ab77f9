"""Hand-placed test scenes (Gaussians at chosen pixel centres and depths)."""
import math

import numpy as np

from paper_2509_25191_gb300.synth import Scene, Views

Y00 = 0.28209479177387814  # degree-0 SH value, for DC coefficients of a colour


def logit(o):
    return math.log(o / (1.0 - o))


def pinhole_views(W, H, f, cx=None, cy=None, viewmat=None, n=1):
    vm = np.concatenate([np.eye(3).reshape(-1), np.zeros(3)]) if viewmat is None else np.asarray(viewmat)
    cx = W / 2.0 if cx is None else cx
    cy = H / 2.0 if cy is None else cy
    return Views(vm.reshape(1, 12).astype(np.float32), np.array([[f, f, cx, cy]], np.float32),
                 np.array([W], np.int32), np.array([H], np.int32),
                 np.array([0], np.int64), np.array([n], np.int64))


def at_pixel(u, v, z, f, cx, cy):
    """World point (camera at identity) projecting to the centre of pixel (u, v)."""
    return np.array([(u + 0.5 - cx) * z / f, (v + 0.5 - cy) * z / f, z])


def make_scene(means, scale, opac, colours, quats=None, sh_degree=0):
    n = len(means)
    means = np.asarray(means, np.float64)
    ls = np.full((n, 3), math.log(scale)) if np.isscalar(scale) else np.log(np.asarray(scale, np.float64))
    q = np.tile([1.0, 0, 0, 0], (n, 1)) if quats is None else np.asarray(quats, np.float64)
    lg = np.array([logit(o) for o in np.broadcast_to(opac, (n,))])
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = (np.asarray(colours, np.float64) - 0.5) / Y00
    return Scene(means.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                 lg.astype(np.float32), sh.astype(np.float32), sh_degree)
