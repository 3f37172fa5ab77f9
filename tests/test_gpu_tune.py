"""The autotuner times each candidate tile shape on the caller's inputs,
returns the fastest, and caches the choice per workload signature."""
import json

import numpy as np
import pytest
import torch

from paper_2509_25191_gb300 import _lib, synth
from paper_2509_25191_gb300.tune import CANDIDATES, autotune

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_and_caches(tmp_path):
    sc, vw = synth.orbit_views(0, 20000, 2, 200, 112, 200.0)
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    target = torch.rand(views.num_image_floats(), device="cuda")
    cache = str(tmp_path / "tune.json")
    best, times = autotune(g, views, target, reps=3, cache_path=cache)
    assert best in CANDIDATES and set(times) == set(CANDIDATES)
    assert times[best] == min(times.values()) and all(np.isfinite(list(times.values())))
    entry = next(iter(json.load(open(cache)).values()))
    assert tuple(entry["tile"]) == best
    again, times2 = autotune(g, views, target, reps=3, cache_path=cache)
    assert again == best and times2 == times
