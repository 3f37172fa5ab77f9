"""Checkpoint round trip of a training run's state (CPU): parameters, pose
residuals, optimiser moments, step and generator states come back equal, and
a failed save leaves the previous checkpoint readable."""
import types

import pytest
import torch

from paper_2509_25191_gb300 import checkpoint


def _state(seed):
    g = torch.Generator().manual_seed(seed)
    r = lambda *s: torch.randn(*s, generator=g)
    gauss = types.SimpleNamespace(means=r(50, 3), log_scales=r(50, 3), quats=r(50, 4), opacity_logits=r(50),
                                  sh=r(50, 16, 3))
    return gauss, {"dr": r(7, 6), "dt": r(7, 3)}, {"means": (r(50, 3), r(50, 3).abs())}


def test_round_trip(tmp_path):
    gauss, pose, opt = _state(0)
    gen = torch.Generator().manual_seed(123)
    torch.randn(5, generator=gen)                      # advance the stream
    path = tmp_path / "ckpt" / "run.pt"
    checkpoint.save(path, gauss, step=4321, pose_residuals=pose, optimizer_state=opt, generators={"noise": gen},
                    extra={"tile": [32, 16]})
    want_next = torch.randn(3, generator=gen)
    gen2 = torch.Generator().manual_seed(999)
    out = checkpoint.load(path, generators={"noise": gen2})
    assert out["step"] == 4321 and out["extra"] == {"tile": [32, 16]}
    for k in checkpoint.GAUSSIAN_FIELDS:
        assert torch.equal(out["gaussians"][k], getattr(gauss, k))
    for k in pose:
        assert torch.equal(out["pose_residuals"][k], pose[k])
    assert torch.equal(out["optimizer"]["means"][0], opt["means"][0])
    assert torch.equal(out["optimizer"]["means"][1], opt["means"][1])
    assert torch.equal(torch.randn(3, generator=gen2), want_next)   # the noise stream resumes where it stopped


def test_interrupted_save_keeps_the_previous_checkpoint(tmp_path, monkeypatch):
    gauss, pose, opt = _state(1)
    path = tmp_path / "run.pt"
    checkpoint.save(path, gauss, step=1, pose_residuals=pose)

    def boom(obj, f):
        open(f, "wb").write(b"partial")
        raise OSError("disk full")

    monkeypatch.setattr(checkpoint.torch, "save", boom)
    with pytest.raises(OSError):
        checkpoint.save(path, gauss, step=2, pose_residuals=pose)
    monkeypatch.undo()
    assert checkpoint.load(path)["step"] == 1
