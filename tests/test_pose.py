"""The per-view residual pose of Section 3.4 (6D rotation representation
and the composition R' = dR R, t' = t + dt), on CPU in float64."""
import numpy as np
import torch

from paper_2509_25191_gb300 import pose


def _random_rotations(n, seed):
    q = np.random.default_rng(seed).standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)


def test_identity_residual_leaves_the_pose_unchanged():
    vm = torch.as_tensor(np.concatenate([_random_rotations(5, 0).reshape(5, 9),
                                         np.random.default_rng(1).standard_normal((5, 3))], 1))
    dr = pose.identity_6d(5, dtype=torch.float64)
    assert torch.equal(pose.rotation_6d(dr), torch.eye(3, dtype=torch.float64).expand(5, 3, 3))
    assert torch.allclose(pose.apply_residual(vm, dr, torch.zeros(5, 3, dtype=torch.float64)), vm, atol=1e-15)


def test_first_two_columns_of_a_rotation_give_it_back():
    R = _random_rotations(16, 2)
    dr = torch.as_tensor(np.concatenate([R[:, :, 0], R[:, :, 1]], 1))
    assert np.allclose(pose.rotation_6d(dr).numpy(), R, atol=1e-12)


def test_any_6d_vector_maps_to_a_proper_rotation():
    dr = torch.as_tensor(np.random.default_rng(3).standard_normal((64, 6)))
    M = pose.rotation_6d(dr).numpy()
    assert np.allclose(M @ np.swapaxes(M, 1, 2), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(M), 1.0, atol=1e-12)
    # the first column follows a1 alone; scaling a1 or adding a multiple of a1 to a2 changes nothing
    a1, a2 = dr[:, :3], dr[:, 3:]
    assert np.allclose(M[:, :, 0], (a1 / a1.norm(dim=1, keepdim=True)).numpy(), atol=1e-12)
    dr2 = torch.cat([2.5 * a1, a2 - 0.7 * a1], 1)
    assert np.allclose(pose.rotation_6d(dr2).numpy(), M, atol=1e-12)


def test_composition_and_gradients():
    rng = np.random.default_rng(4)
    R = _random_rotations(3, 5)
    t = rng.standard_normal((3, 3))
    vm = torch.as_tensor(np.concatenate([R.reshape(3, 9), t], 1))
    dr = torch.as_tensor(rng.standard_normal((3, 6))).requires_grad_(True)
    dt = torch.as_tensor(rng.standard_normal((3, 3))).requires_grad_(True)
    out = pose.apply_residual(vm, dr, dt).detach().numpy()
    dR = pose.rotation_6d(dr).detach().numpy()
    assert np.allclose(out[:, :9].reshape(3, 3, 3), dR @ R, atol=1e-14)
    assert np.allclose(out[:, 9:], t + dt.detach().numpy(), atol=1e-15)
    assert torch.autograd.gradcheck(lambda a, b: pose.apply_residual(vm, a, b), (dr, dt), eps=1e-6, atol=1e-8)


def test_pose_learning_rate_schedule():
    """Section 4.1: 1e-4 at the start, decayed exponentially to a tenth over
    the run (geometric mean half way), flat after the end."""
    assert pose.pose_lr(0) == 1e-4
    assert np.isclose(pose.pose_lr(30000), 1e-5, rtol=1e-12)
    assert np.isclose(pose.pose_lr(15000), 1e-4 * 0.1 ** 0.5, rtol=1e-12)
    assert np.isclose(pose.pose_lr(45000), 1e-5, rtol=1e-12)
    lrs = [pose.pose_lr(k, total_steps=100) for k in range(101)]
    ratios = np.array(lrs[1:]) / np.array(lrs[:-1])
    assert np.allclose(ratios, 0.1 ** 0.01, rtol=1e-12)   # constant ratio: exponential
