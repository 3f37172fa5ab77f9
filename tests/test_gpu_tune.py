"""The autotuner times (tile, shared-memory batch) candidates on the caller's
inputs, returns the fastest, and caches the choice per workload signature;
every candidate renders the same image bit for bit and the same gradients
up to the order of float additions."""
import json

import numpy as np
import pytest
import torch

from paper_2509_25191_gb300 import _lib, synth
from paper_2509_25191_gb300.autograd import Rasterizer
from paper_2509_25191_gb300.tune import Choice, autotune, candidates, key_str

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_candidate_and_caches(tmp_path):
    sc, vw = synth.orbit_views(0, 20000, 2, 200, 112, 200.0)
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    target = torch.rand(views.num_image_floats(), device="cuda")
    cache = str(tmp_path / "tune.json")
    best, times = autotune(g, views, target, reps=3, cache_path=cache)
    assert best in candidates() and set(times) <= set(candidates()) and len(times) >= 6 + 2 * 4
    assert times[best] == min(times.values()) and all(np.isfinite(list(times.values())))
    entry = next(iter(json.load(open(cache)).values()))
    assert entry["best"] == key_str(best)
    again, times2 = autotune(g, views, target, reps=3, cache_path=cache)
    assert again == best and times2 == times


@pytest.mark.parametrize("case", ["orbit", "clustered"])
def test_every_tile_and_batch_renders_the_same_image(case):
    if case == "orbit":
        sc, vw = synth.orbit_views(0, 20000, 3, 200, 112, 200.0)
    else:
        sc = synth.cluster_scene(0, 30000)
        vw = synth._views(synth.look_at((0.0, 0.0, -6.0)), 1000.0 * 333 / 1237.0, 333, 221, 0, 30000)
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    up = torch.randn(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    ref_img = ref_g2d = None
    for c in candidates():
        rast = Rasterizer(tile=c.tile, batch=c.batch)
        image, proj = rast.forward(g, views)
        g2d = torch.empty(max(1, views.num_slots()), _lib.GS_GRAD2D_FLOATS, device="cuda")
        _lib.gs_rasterize_bwd(views, rast.cfg, proj, rast.bins, image, up, g2d)
        torch.cuda.synchronize()
        rast.check_status()
        img, gg = image.cpu().numpy(), g2d.cpu().numpy()
        if ref_img is None:
            ref_img, ref_g2d = img, gg
            continue
        assert np.array_equal(img.view(np.uint32), ref_img.view(np.uint32)), key_str(c)
        assert np.linalg.norm(gg - ref_g2d) <= 1e-5 * np.linalg.norm(ref_g2d), key_str(c)
