"""Pins of the FP64 pose-residual oracle (Section 3.4: 6D rotation residual
and translation residual, R' = dR R, t' = t + dt) against facts the
mathematics fixes, and planted mistakes that each of them catches."""
import numpy as np
import pytest

from oracle import pose as P


def _rotations(n, seed):
    """Random rotations from normalised quaternions (Hamilton convention),
    built independently of the 6D map."""
    q = np.random.default_rng(seed).standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def _viewmats(n, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([_rotations(n, seed + 100).reshape(n, 9), rng.standard_normal((n, 3))], 1)


# --------------------------------------------------------------------------
# pins, written against an implementation (rot6d, apply, vjp) so that the
# planted-mistake test below can run them on a broken copy
# --------------------------------------------------------------------------

def pin_columns_give_rotation_back(rot6d, apply, vjp):
    R = _rotations(16, 2)
    got = rot6d(np.concatenate([R[:, :, 0], R[:, :, 1]], 1))
    return np.allclose(got, R, atol=1e-12)


def pin_axis_rotations(rot6d, apply, vjp):
    """Rotation by theta about z, x and y (right-handed, columns are the
    images of the basis vectors), given by a scaled first column and a second
    column with a multiple of the first added."""
    ok = True
    for th in (0.3, -1.2, 2.9):
        c, s = np.cos(th), np.sin(th)
        Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
        Rx = np.array([[1.0, 0, 0], [0, c, -s], [0, s, c]])
        Ry = np.array([[c, 0, s], [0, 1.0, 0], [-s, 0, c]])
        for R in (Rz, Rx, Ry):
            a1 = 3.7 * R[:, 0]
            a2 = R[:, 1] - 0.8 * R[:, 0]
            ok &= np.allclose(rot6d(np.concatenate([a1, a2])), R, atol=1e-13)
    return ok


def pin_proper_rotation(rot6d, apply, vjp):
    a = np.random.default_rng(3).standard_normal((64, 6))
    M = rot6d(a)
    ok = np.allclose(M @ np.swapaxes(M, 1, 2), np.eye(3), atol=1e-12)
    ok &= np.allclose(np.linalg.det(M), 1.0, atol=1e-12)
    ok &= np.allclose(M[:, :, 0], a[:, :3] / np.linalg.norm(a[:, :3], axis=1, keepdims=True), atol=1e-12)
    # the second column lies in the plane of a1 and a2, on a2's side of a1
    ok &= bool(np.all(np.einsum("vi,vi->v", M[:, :, 1], a[:, 3:]) > 0))
    return ok


def pin_identity_and_translation(rot6d, apply, vjp):
    vm = _viewmats(5, 1)
    ok = np.allclose(apply(vm, P.identity_6d(5), np.zeros((5, 3))), vm, atol=1e-15)
    # a pure translation residual moves the camera centre C = -R^T t by -R^T dt
    dt = np.random.default_rng(9).standard_normal((5, 3))
    out = apply(vm, P.identity_6d(5), dt)
    R = vm[:, :9].reshape(5, 3, 3)
    C0 = -np.einsum("vji,vj->vi", R, vm[:, 9:])
    C1 = -np.einsum("vji,vj->vi", out[:, :9].reshape(5, 3, 3), out[:, 9:])
    ok &= np.allclose(C1 - C0, -np.einsum("vji,vj->vi", R, dt), atol=1e-12)
    return ok


def pin_left_composition(rot6d, apply, vjp):
    """A residual acts on the camera frame (left): applying dr1 then dr2 is
    the rotation dR2 dR1 R, and a rotation residual alone leaves t as it is."""
    rng = np.random.default_rng(4)
    vm = _viewmats(3, 5)
    d1, d2 = rng.standard_normal((3, 6)), rng.standard_normal((3, 6))
    z = np.zeros((3, 3))
    out = apply(apply(vm, d1, z), d2, z)
    R = vm[:, :9].reshape(3, 3, 3)
    want = rot6d(d2) @ rot6d(d1) @ R
    return np.allclose(out[:, :9].reshape(3, 3, 3), want, atol=1e-13) and np.allclose(out[:, 9:], vm[:, 9:])


def pin_vjp_central_differences(rot6d, apply, vjp):
    rng = np.random.default_rng(11)
    ok = True
    for case in range(3):
        vm = _viewmats(4, 20 + case)
        dr = P.identity_6d(4) if case == 0 else rng.standard_normal((4, 6))
        dt = np.zeros((4, 3)) if case == 0 else rng.standard_normal((4, 3))
        W = rng.standard_normal((4, 12))
        g_dr, g_dt = vjp(vm, dr, dt, W)
        h = 1e-6
        fd_dr = np.zeros_like(dr)
        fd_dt = np.zeros_like(dt)
        for v in range(4):
            for k in range(6):
                e = np.zeros_like(dr)
                e[v, k] = h
                fd_dr[v, k] = (np.sum(W * apply(vm, dr + e, dt)) - np.sum(W * apply(vm, dr - e, dt))) / (2 * h)
            for k in range(3):
                e = np.zeros_like(dt)
                e[v, k] = h
                fd_dt[v, k] = (np.sum(W * apply(vm, dr, dt + e)) - np.sum(W * apply(vm, dr, dt - e))) / (2 * h)
        ok &= np.allclose(g_dr, fd_dr, rtol=1e-6, atol=1e-8) and np.allclose(g_dt, fd_dt, rtol=1e-6, atol=1e-8)
    return ok


PINS = [pin_columns_give_rotation_back, pin_axis_rotations, pin_proper_rotation, pin_identity_and_translation,
        pin_left_composition, pin_vjp_central_differences]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    assert pin(P.rotation_6d, P.apply_residual, P.residual_vjp)


# --------------------------------------------------------------------------
# planted mistakes: each broken copy must fail at least one pin
# --------------------------------------------------------------------------

def _rot6d_swapped_cross(a):
    M = P.rotation_6d(a)
    M[..., 2] = -M[..., 2]            # b3 = b2 x b1
    return M


def _rot6d_rows(a):
    return np.swapaxes(P.rotation_6d(a), -1, -2)   # b1, b2, b3 as rows


def _rot6d_no_orthogonalisation(a):
    a = np.asarray(a, np.float64).reshape(-1, 6)
    out = []
    for v in a:
        b1 = v[:3] / np.linalg.norm(v[:3])
        b2 = v[3:] / np.linalg.norm(v[3:])   # a2 not made orthogonal to b1
        out.append(np.stack([b1, b2, np.cross(b1, b2)], 1))
    out = np.array(out)
    return out[0] if out.shape[0] == 1 and np.asarray(a).ndim == 1 else out


def _apply_right(vm, dr, dt):
    vm = np.asarray(vm, np.float64).reshape(-1, 12)
    out = vm.copy()
    for v in range(vm.shape[0]):
        out[v, :9] = (vm[v, :9].reshape(3, 3) @ P.rotation_6d(np.asarray(dr).reshape(-1, 6)[v])).reshape(-1)
        out[v, 9:] = vm[v, 9:] + np.asarray(dt).reshape(-1, 3)[v]
    return out


def _apply_rotated_translation(vm, dr, dt):
    vm = np.asarray(vm, np.float64).reshape(-1, 12)
    out = P.apply_residual(vm, dr, dt)
    for v in range(vm.shape[0]):
        dR = P.rotation_6d(np.asarray(dr).reshape(-1, 6)[v])
        out[v, 9:] = dR @ vm[v, 9:] + np.asarray(dt).reshape(-1, 3)[v]   # t' = dR t + dt
    return out


def _vjp_transposed_G(vm, dr, dt, g):
    gt = np.asarray(g, np.float64).reshape(-1, 12).copy()
    R = np.asarray(vm, np.float64).reshape(-1, 12)[:, :9].reshape(-1, 3, 3)
    # R^T dL/dR' instead of dL/dR' R^T: feed a gradient that yields it
    G_wrong = np.swapaxes(R, 1, 2) @ gt[:, :9].reshape(-1, 3, 3)
    gt[:, :9] = (G_wrong @ R).reshape(-1, 9)
    return P.residual_vjp(vm, dr, dt, gt)


def _vjp_without_cross_term(vm, dr, dt, g):
    d_dr, d_dt = P.residual_vjp(vm, dr, dt, g)
    return d_dr * np.array([1, 1, 1, 0.5, 0.5, 0.5]), d_dt


def _vjp_sign_of_translation(vm, dr, dt, g):
    d_dr, d_dt = P.residual_vjp(vm, dr, dt, g)
    return d_dr, -d_dt


MISTAKES = {
    "b3 = b2 x b1": (_rot6d_swapped_cross, P.apply_residual, P.residual_vjp),
    "columns written as rows": (_rot6d_rows, P.apply_residual, P.residual_vjp),
    "no Gram-Schmidt step": (_rot6d_no_orthogonalisation, P.apply_residual, P.residual_vjp),
    "right composition R dR": (P.rotation_6d, _apply_right, P.residual_vjp),
    "translation rotated by dR": (P.rotation_6d, _apply_rotated_translation, P.residual_vjp),
    "transposed chain through R": (P.rotation_6d, P.apply_residual, _vjp_transposed_G),
    "a2 gradient halved": (P.rotation_6d, P.apply_residual, _vjp_without_cross_term),
    "translation gradient sign": (P.rotation_6d, P.apply_residual, _vjp_sign_of_translation),
}


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_mistake_fails_a_pin(name):
    impl = MISTAKES[name]
    failed = []
    for pin in PINS:
        try:
            ok = pin(*impl)
        except (ValueError, IndexError, np.linalg.LinAlgError):
            ok = False
        if not ok:
            failed.append(pin.__name__)
    assert failed, f"planted mistake '{name}' passes every pin"


def test_agrees_with_the_alignment_oracle_residual_chain():
    """Third opinion: the global-alignment oracle states the same residual
    (with a focal term) and its own chain rule; with the focal term off the
    two give the same cameras and the same gradients."""
    from oracle import ga as GA
    rng = np.random.default_rng(30)
    vm = _viewmats(6, 31)
    dr = rng.standard_normal((6, 6))
    dt = rng.standard_normal((6, 3))
    W = rng.standard_normal((6, 12))
    intr = np.tile([1000.0, 1000.0, 500.0, 400.0], (6, 1))
    res = np.concatenate([dr, dt, np.zeros((6, 1))], 1)
    _, vm_ga = GA.apply_residuals(intr, vm, res, optimise_focal=False)
    assert np.allclose(vm_ga, P.apply_residual(vm, dr, dt), atol=1e-14)
    g_ga = GA.residual_vjp(intr, vm, res, np.zeros((6, 4)), W, optimise_focal=False)
    d_dr, d_dt = P.residual_vjp(vm, dr, dt, W)
    assert np.allclose(g_ga[:, :6], d_dr, atol=1e-12) and np.allclose(g_ga[:, 6:9], d_dt, atol=1e-14)
