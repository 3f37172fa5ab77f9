"""The spatial-order helper: Morton codes bit-exact against a numpy
statement of their definition, and a reordered scene renders the same image
with its gradients permuted the same way."""
import numpy as np
import pytest
import torch

from paper_2509_25191_gb300 import _lib, synth
from paper_2509_25191_gb300.autograd import Rasterizer
from paper_2509_25191_gb300.layout import reorder, spatial_order

pytestmark = pytest.mark.gpu


def _morton_ref(m, lo, hi):
    """float32 quantisation exactly as stated (scale 2^21 / (hi - lo) rounded
    to float32, then (m - lo) * scale in float32), bits interleaved x y z."""
    m = m.astype(np.float32)
    lo = np.asarray(lo, np.float32)
    scale = (np.float32(2097152.0) / (np.asarray(hi, np.float32) - lo)).astype(np.float32)
    t = ((m - lo).astype(np.float32) * scale).astype(np.float32)
    q = np.where(t > 0, np.minimum(np.floor(t), 2097151), 0).astype(np.uint64)
    code = np.zeros(len(m), np.uint64)
    for b in range(21):
        for a in range(3):
            code |= ((q[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + a)
    return code


def test_codes_match_the_definition():
    rng = np.random.default_rng(0)
    m = rng.normal(0, 2, (100_003, 3)).astype(np.float32)
    m[5] = [np.nan, 0, 0]
    m[7] = [np.inf, 0, 0]
    lo, hi = [-3.0, -4.0, -5.0], [3.0, 4.0, 5.0]   # some means outside the box on both sides
    codes = torch.empty(len(m), dtype=torch.int64, device="cuda")
    _lib.gs_spatial_codes(torch.as_tensor(m).cuda(), lo + hi, codes)
    got = codes.cpu().numpy().view(np.uint64)
    want = _morton_ref(m, lo, hi)
    want[[5, 7]] = np.iinfo(np.uint64).max
    assert np.array_equal(got, want)


def test_reordered_scene_renders_the_same_image_and_permuted_gradients():
    sc, vw = synth.orbit_views(1, 20000, 3, 160, 96, 1000.0 * 160 / 979.0)
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    perm = spatial_order(g.means)
    assert sorted(perm.cpu().tolist()) == list(range(g.n)) and not torch.equal(perm, torch.arange(g.n).cuda())
    gp = reorder(g, perm)
    up = torch.randn(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    outs = []
    for gg in (g, gp):
        rast = Rasterizer(tile=(16, 16))
        image, proj = rast.forward(gg, views)
        grads, dvm, _ = rast.backward(gg, views, proj, image, up)
        torch.cuda.synchronize()
        outs.append((image.cpu().numpy(), grads.means.clone(), dvm.cpu().numpy()))
    # the same image up to the order of Gaussians at exactly equal float32
    # depths (ties follow the index, which the permutation changes)
    assert np.abs(outs[0][0] - outs[1][0]).max() <= 1e-6
    a = outs[0][1][perm].cpu().numpy()
    b = outs[1][1].cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a)
    assert np.linalg.norm(outs[0][2] - outs[1][2]) <= 1e-5 * np.linalg.norm(outs[0][2])


def test_ranges_keep_each_scene_in_place():
    sc, vw = synth.uneven_scenes(seeds=(1, 2), sizes=(300, 500), views_per_scene=1, resolutions=((64, 48),))
    means = torch.as_tensor(sc.means).cuda()
    perm = spatial_order(means, ranges=[(0, 300), (300, 500)]).cpu().numpy()
    assert sorted(perm[:300]) == list(range(300)) and sorted(perm[300:]) == list(range(300, 800))
