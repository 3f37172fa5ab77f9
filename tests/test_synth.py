"""Input generators: deterministic, shaped as the workloads state."""
import numpy as np

from paper_2509_25191_gb300 import synth


def test_generators_are_deterministic():
    a, va = synth.single_view_small()
    b, vb = synth.single_view_small()
    for k in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        assert np.array_equal(getattr(a, k), getattr(b, k))
    assert np.array_equal(va.viewmats, vb.viewmats)


def test_small_config_shapes_and_ranges():
    sc, vw = synth.single_view_small()
    assert sc.n == 2000 and sc.sh.shape == (2000, 1, 3)
    assert (sc.means[:, :2] >= -1).all() and (sc.means[:, :2] <= 1).all()
    assert (sc.means[:, 2] >= 2).all() and (sc.means[:, 2] <= 4).all()
    assert np.allclose(np.linalg.norm(sc.quats, axis=1), 1, atol=1e-6)
    assert vw.width[0] == 128 and vw.intrinsics[0, 0] == 150 and vw.intrinsics[0, 2] == 64


def test_orbit_cameras_look_at_origin():
    vm = synth.orbit_viewmats(16)
    for m in vm:
        R, t = m[:9].reshape(3, 3), m[9:]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12)
        c = -R.T @ t
        assert abs(np.linalg.norm(c) - 5) < 1e-9 and abs(c[1]) < 1e-12
        # the origin projects to the principal point
        assert np.allclose((R @ np.zeros(3) + t)[:2], 0, atol=1e-9)


def test_uneven_scene_layout():
    sc, vw = synth.uneven_scenes(sizes=(100, 200, 300), seeds=(1, 2, 3))
    assert sc.n == 600 and vw.n == 12
    assert list(vw.gauss_begin) == [0] * 4 + [100] * 4 + [300] * 4
    assert list(vw.gauss_count) == [100] * 4 + [200] * 4 + [300] * 4


def test_jitter_is_one_degree_and_one_percent():
    mats = synth.hemisphere_viewmats(10)
    jit = synth.jitter_viewmats(mats, 0)
    for a, b in zip(mats, jit):
        Ra, Rb = a[:9].reshape(3, 3), b[:9].reshape(3, 3)
        ang = np.degrees(np.arccos(np.clip((np.trace(Rb @ Ra.T) - 1) / 2, -1, 1)))
        assert abs(ang - 1.0) < 1e-6
        assert abs(np.linalg.norm(b[9:] - a[9:]) - 0.01 * np.linalg.norm(a[9:])) < 1e-9
