"""FP64 statement of the per-view residual pose of Section 3.4.

TEST INFRASTRUCTURE ONLY: imported by the tests and never by the product
package. It shares no code with the CUDA library or with the product's torch
residual map.

Section 3.4 refines every camera by a translation residual dt in R^3 and a
rotation residual in the 6D representation of Zhou et al. (two 3-vectors
a1, a2 turned into a rotation by Gram-Schmidt). The refined world->camera
pose is R' = dR R, t' = t + dt (left composition; the residual starts at
a1 = (1,0,0), a2 = (0,1,0), dt = 0, which leaves the pose unchanged).

Functions and what pins them (tests/test_oracle_pose.py):

* ``rotation_6d``     -- the two leading columns of any rotation give it back;
                         every 6D vector maps to a proper rotation (orthonormal,
                         det +1); the first column depends on a1 alone and the
                         map ignores the scale of a1 and any multiple of a1
                         added to a2 (the Gram-Schmidt invariances); Rodrigues
                         rotations about the coordinate axes.
* ``apply_residual``  -- identity residual leaves the pose unchanged; a pure
                         translation residual moves the camera centre by
                         -R^T dt; the composition of two residuals.
* ``residual_vjp``    -- FP64 central differences of ``apply_residual``, on
                         random residuals far from the identity and at it.
"""
from __future__ import annotations

import numpy as np


def rotation_6d(a):
    """[6] or [V,6] -> [3,3] or [V,3,3]: columns b1 = a1/|a1|,
    b2 = (a2 - (b1.a2) b1)/|a2 - (b1.a2) b1|, b3 = b1 x b2."""
    a = np.asarray(a, np.float64)
    single = a.ndim == 1
    a = a.reshape(-1, 6)
    out = np.empty((a.shape[0], 3, 3))
    for v in range(a.shape[0]):
        a1, a2 = a[v, :3], a[v, 3:]
        b1 = a1 / np.sqrt(a1 @ a1)
        u = a2 - (b1 @ a2) * b1
        b2 = u / np.sqrt(u @ u)
        b3 = np.array([b1[1] * b2[2] - b1[2] * b2[1], b1[2] * b2[0] - b1[0] * b2[2], b1[0] * b2[1] - b1[1] * b2[0]])
        out[v, :, 0], out[v, :, 1], out[v, :, 2] = b1, b2, b3
    return out[0] if single else out


def identity_6d(n):
    return np.tile(np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.0]), (n, 1))


def apply_residual(viewmats, dr, dt):
    """viewmats [V,12] (R row-major, then t) -> [V,12] with R' = dR R,
    t' = t + dt, dR = rotation_6d(dr)."""
    vm = np.asarray(viewmats, np.float64).reshape(-1, 12)
    dr = np.asarray(dr, np.float64).reshape(-1, 6)
    dt = np.asarray(dt, np.float64).reshape(-1, 3)
    out = np.empty_like(vm)
    for v in range(vm.shape[0]):
        R = vm[v, :9].reshape(3, 3)
        out[v, :9] = (rotation_6d(dr[v]) @ R).reshape(-1)
        out[v, 9:] = vm[v, 9:] + dt[v]
    return out


def residual_vjp(viewmats, dr, dt, dL_dvm):
    """Gradients (dL/d dr [V,6], dL/d dt [V,3]) of L through
    apply_residual(viewmats, dr, dt), given dL/d(R', t') = dL_dvm [V,12]
    (dL/dR' row-major, then dL/dt'), by the chain rule written out:

      R' = dR R            -> G = dL/d dR = dL/dR' R^T, columns g1 g2 g3
      b3 = b1 x b2         -> dL/db1 += b2 x g3,  dL/db2 += g3 x b1
      b2 = u / |u|         -> dL/du = (dL/db2 - b2 (b2 . dL/db2)) / |u|
      u = a2 - (b1.a2) b1  -> dL/da2 = dL/du - (b1 . dL/du) b1,
                              dL/db1 += -(b1.a2) dL/du - (b1 . dL/du) a2
      b1 = a1 / |a1|       -> dL/da1 = (dL/db1 - b1 (b1 . dL/db1)) / |a1|
      t' = t + dt          -> dL/d dt = dL/dt'
    """
    vm = np.asarray(viewmats, np.float64).reshape(-1, 12)
    dr = np.asarray(dr, np.float64).reshape(-1, 6)
    g = np.asarray(dL_dvm, np.float64).reshape(-1, 12)
    d_dr = np.zeros_like(dr)
    d_dt = g[:, 9:].copy()
    for v in range(vm.shape[0]):
        a1, a2 = dr[v, :3], dr[v, 3:]
        n1 = np.sqrt(a1 @ a1)
        b1 = a1 / n1
        s = b1 @ a2
        u = a2 - s * b1
        nu = np.sqrt(u @ u)
        b2 = u / nu
        G = g[v, :9].reshape(3, 3) @ vm[v, :9].reshape(3, 3).T
        gb1, gb2, gb3 = G[:, 0].copy(), G[:, 1].copy(), G[:, 2].copy()
        gb1 += np.cross(b2, gb3)
        gb2 += np.cross(gb3, b1)
        gu = (gb2 - b2 * (b2 @ gb2)) / nu
        d_dr[v, 3:] = gu - (b1 @ gu) * b1
        gb1 += -s * gu - (b1 @ gu) * a2
        d_dr[v, :3] = (gb1 - b1 * (b1 @ gb1)) / n1
    return d_dr, d_dt
