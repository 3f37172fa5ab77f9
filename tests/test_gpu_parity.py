"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2509_25191_gb300 import _lib, synth
from paper_2509_25191_gb300.autograd import Rasterizer
from tests.gpu_util import (check_grad, conic_to_cov_grads, gpu_forward, image_errors, oracle_forward, split,
                            upstream)

pytestmark = pytest.mark.gpu


def _eye_view(n, W, H, f, cx=None, cy=None):
    return synth._views(np.concatenate([np.eye(3).reshape(-1), np.zeros(3)]), f, W, H, 0, n) if cx is None else \
        synth.Views(np.concatenate([np.eye(3).reshape(-1), np.zeros(3)]).reshape(1, 12).astype(np.float32),
                    np.array([[f, f, cx, cy]], np.float32), np.array([W], np.int32), np.array([H], np.int32),
                    np.array([0]), np.array([n]))


def _reduced_c2(n=30000, W=333, H=221, seed=0):
    """The 1M-Gaussian clustered SH3 workload scaled down: same distributions,
    fewer Gaussians, lower resolution (ragged tiles on both axes)."""
    sc = synth.cluster_scene(seed, n)
    vw = synth._views(synth.look_at((0.0, 0.0, -6.0)), 1000.0 * W / 1237.0, W, H, 0, n)
    return sc, vw


CASES = {
    "small_2k": lambda: synth.single_view_small(),
    "clustered_sh3": lambda: _reduced_c2(),
    "orbit_4views": lambda: synth.orbit_views(0, 20000, 4, 200, 112, 1000.0 * 200 / 979.0),
    "uneven_3scenes": lambda: synth.uneven_scenes(seeds=(1, 2, 3), sizes=(3000, 6000, 9000), views_per_scene=2,
                                                  resolutions=((96, 64), (150, 90), (77, 131)), focal=150.0),
    # the view sees Gaussians [37, 11939) of 12,000: the first 37 and last 61
    # get zero gradients, and the staged projection blocks start mid-array
    "subset_view": lambda: (synth.cluster_scene(4, 12000),
                            synth._views(synth.look_at((0.0, 0.0, -6.0)), 1000.0 * 300 / 1237.0, 300, 200, 37,
                                         12000 - 37 - 61)),
}


# ---------------------------------------------------------------------------
# library / ABI
# ---------------------------------------------------------------------------

def test_invalid_arguments_rejected_on_host():
    sc, vw = synth.single_view_small(n=50)
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    proj = torch.empty(50, 16, device="cuda")
    with pytest.raises(_lib.GsError) as e:
        _lib.gs_project(g, views, _lib.config(tile=(12, 16)), proj)
    assert e.value.code == _lib.GS_ERR_UNSUPPORTED
    bad = _lib.Views(views.viewmats, views.intrinsics, [128], [128], [0], [51])   # range past n
    with pytest.raises(_lib.GsError) as e:
        _lib.gs_project(g, bad, _lib.config(), proj)
    assert e.value.code == _lib.GS_ERR_ARG
    buf = torch.empty(50 * 16 + 4, device="cuda")
    with pytest.raises(_lib.GsError) as e:
        _lib.gs_project(g, views, _lib.config(), buf[1:1 + 50 * 16])   # 4-byte offset: not 16-byte aligned
    assert e.value.code == _lib.GS_ERR_ARG
    sc4 = synth.uniform_box_scene(0, 50, sh_degree=3)
    sc4.sh = np.zeros((50, 25, 3), np.float32)                           # degree 4 is not supported
    g4 = _lib.Gaussians.__new__(_lib.Gaussians)
    g4.__dict__.update(g.__dict__)
    g4.sh_degree = 4
    with pytest.raises(_lib.GsError) as e:
        _lib.gs_project(g4, views, _lib.config(), proj)
    assert e.value.code == _lib.GS_ERR_UNSUPPORTED
    torch.cuda.synchronize()


def test_capacity_overflow_reports_needed_count():
    sc, vw = synth.single_view_small()
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    rast = Rasterizer()
    proj = rast.project(g, views)
    cfg = rast.cfg
    small = _lib.Bins(views.num_tiles(cfg), 10)
    status = _lib.new_status()
    _lib.gs_bin_sort(views, cfg, proj, small, status)
    img = torch.empty(views.num_image_floats(), device="cuda")
    _lib.gs_render_fwd(views, cfg, proj, small, img, status)
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    need = int(small.counters[0].item())
    assert st[0] == _lib.GS_ERR_CAPACITY and st[1] == need and need > 10
    assert float(img.abs().max()) == 0.0
    # a big enough capacity works afterwards in the same context
    image, _ = rast.forward(g, views)
    torch.cuda.synchronize()
    rast.check_status()
    assert rast.last_instances == need


# ---------------------------------------------------------------------------
# projection
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["small_2k", "clustered_sh3", "orbit_4views"])
def test_projection_parity(case):
    sc, vw = CASES[case]()
    _, _, views, _, proj = gpu_forward(sc, vw)
    P = proj.cpu().numpy()
    for v in range(vw.n):
        ref = O.project_view(sc, vw, v)
        rec = P[views.slot_base(v): views.slot_base(v) + int(vw.gauss_count[v])]
        rad = rec[:, 11]
        both = (rad > 0) & (ref["radius"] > 0)
        # validity agrees except where the radius itself is ambiguous
        frac = ref["r_real"] - np.floor(ref["r_real"])
        amb = (frac < 1e-4) | (frac > 1 - 1e-4)
        disagree = ((rad > 0) != (ref["radius"] > 0)) & ~amb
        assert disagree.sum() <= max(2, 1e-4 * len(rad)), disagree.sum()
        x = rec[:, 0].astype(np.float64) + rec[:, 12]
        y = rec[:, 1].astype(np.float64) + rec[:, 13]
        assert np.abs(x - ref["xy"][:, 0])[both].max() < 2e-5 * max(1.0, np.abs(ref["xy"][both]).max())
        assert np.abs(y - ref["xy"][:, 1])[both].max() < 2e-5 * max(1.0, np.abs(ref["xy"][both]).max())
        # the record holds the conic in the staged form; map it back to the
        # covariance (a well-conditioned direction) in FP64
        Ah, beta, Dh = (rec[:, 4:7][both].astype(np.float64)).T
        c = -1.0 / (2.0 * np.log(2.0) * Dh)
        A = -2.0 * np.log(2.0) * Ah
        b = -beta * c
        a = 1.0 / A + b * b / c
        cov = np.stack([a, b, c], 1)
        rc = ref["cov"][both]
        scale = np.abs(rc).max(axis=1, keepdims=True)
        assert (np.abs(cov - rc) / scale).max() < 1e-5
        assert np.abs(rec[:, 7][both] - ref["opac"][both]).max() < 1e-6
        assert np.abs(rec[:, 8:11][both] - ref["rgb"][both]).max() < 1e-5
        ok_r = both & ~amb
        assert np.array_equal(rad[ok_r], ref["radius"][ok_r].astype(np.float32))
        assert np.abs(rec[:, 14][both] / ref["depth"][both] - 1).max() < 1e-6
        # reach extents: the float32 value is enlarged by 2^-14 unless clipped to the radius
        ext, rext = rec[:, 2:4][ok_r], ref["ext"][ok_r]
        assert (ext >= rext * (1 - 1e-6)).all() and (ext <= rext * (1 + 2e-4) + 1e-5).all()


@pytest.mark.parametrize("case", ["clustered_sh3", "orbit_4views", "uneven_3scenes", "subset_view"])
def test_projection_staged_path_equals_per_thread_path(case):
    """Degree 3 stages each full block's SH rows and records with tensor
    copies (swizzled boxes); blocks that straddle scenes, the tail block and
    the fallback read and write per thread. Both give the same records, bit
    for bit (the same arithmetic in the same order)."""
    sc, vw = CASES[case]()
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    cfg = _lib.config()
    n_slots = int(np.sum(vw.gauss_count))
    a = torch.full((n_slots, 16), float("nan"), device="cuda")
    b = torch.full((n_slots, 16), float("nan"), device="cuda")
    status = _lib.new_status()
    _lib.gs_project(g, views, cfg, a, status)
    _lib.gs_project(g, views, _lib.config(use_tma=False), b, status)
    torch.cuda.synchronize()
    assert int(status[0].item()) == 0
    A, B = a.cpu().numpy(), b.cpu().numpy()
    assert not np.isnan(A).any() and np.array_equal(A.view(np.uint32), B.view(np.uint32))


# ---------------------------------------------------------------------------
# binning: bit-exact when fed the oracle's float32 records
# ---------------------------------------------------------------------------

def _records_from_oracle(sc, vw):
    recs = []
    for v in range(vw.n):
        ref = O.project_view(sc, vw, v)
        r = np.zeros((int(vw.gauss_count[v]), 16), np.float32)
        r[:, 0] = ref["xy"][:, 0].astype(np.float32)
        r[:, 1] = ref["xy"][:, 1].astype(np.float32)
        r[:, 11] = ref["radius"].astype(np.float32)
        r[:, 14] = ref["depth"].astype(np.float32)
        r[:, 2:4] = ref["ext"].astype(np.float32)
        recs.append((ref, r))
    return recs


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
@pytest.mark.parametrize("case", ["small_2k", "orbit_4views", "uneven_3scenes"])
def test_binning_bit_exact(case, tile):
    sc, vw = CASES[case]()
    recs = _records_from_oracle(sc, vw)
    proj = torch.as_tensor(np.concatenate([r for _, r in recs])).cuda()
    views = _lib.Views.from_synth(vw)
    cfg = _lib.config(tile=tile)
    n_inst = 0
    refs = []
    for v, (ref, r) in enumerate(recs):
        W, H = int(vw.width[v]), int(vw.height[v])
        refs.append(O.bin_view(r[:, 0], r[:, 1], ref["radius"], r[:, 14], W, H, *tile, ext=r[:, 2:4]))
        n_inst += len(refs[-1][2])
    bins = _lib.Bins(views.num_tiles(cfg), n_inst)
    status = _lib.new_status()
    _lib.gs_bin_sort(views, cfg, proj, bins, status)
    torch.cuda.synchronize()
    assert status[0].item() == 0 and bins.counters[0].item() == n_inst
    ranges = bins.tile_ranges.cpu().numpy().reshape(-1, 2)
    keys = bins.keys.cpu().numpy().view(np.uint64)
    ids = bins.ids.cpu().numpy().view(np.uint32)
    inst_base = 0
    for v, (rr, kk, ii) in enumerate(refs):
        tb = views.tile_base(cfg, v)
        sb = views.slot_base(v)
        G = rr.shape[0]
        got = ranges[tb:tb + G].astype(np.int64) - inst_base
        assert np.array_equal(got, rr)
        sl = slice(inst_base, inst_base + len(ii))
        assert np.array_equal(ids[sl].astype(np.int64) - sb, ii.astype(np.int64))
        exp_keys = (kk & np.uint64(0xffffffff00000000)) | (kk & np.uint64(0xffffffff)) + np.uint64(sb)
        assert np.array_equal(keys[sl], exp_keys)
        inst_base += len(ii)


def test_binning_without_reservation_table_bit_exact():
    """A sparse view on a large tile grid with an exact-size instance buffer:
    the count kernel's reservation table (kept in keys_tmp) does not fit, so
    the scatter counts again and reserves per (block, tile) itself. Same
    bit-exact result."""
    sc, _ = synth.single_view_small(seed=3, n=300)
    vw = _eye_view(300, 1024, 1024, 150.0, 512.0, 512.0)
    recs = _records_from_oracle(sc, vw)
    ref, r = recs[0]
    tile = (16, 16)
    rr, kk, ii = O.bin_view(r[:, 0], r[:, 1], ref["radius"], r[:, 14], 1024, 1024, *tile, ext=r[:, 2:4])
    n_inst = len(ii)
    n_tiles = (1024 // 16) ** 2
    assert 0 < n_inst and n_inst * 8 < n_tiles * 4   # the one-block table would need n_tiles ints
    proj = torch.as_tensor(r).cuda()
    views = _lib.Views.from_synth(vw)
    cfg = _lib.config(tile=tile)
    bins = _lib.Bins(views.num_tiles(cfg), n_inst)
    status = _lib.new_status()
    _lib.gs_bin_sort(views, cfg, proj, bins, status)
    torch.cuda.synchronize()
    assert status[0].item() == 0 and bins.counters[0].item() == n_inst
    assert np.array_equal(bins.tile_ranges.cpu().numpy().reshape(-1, 2).astype(np.int64), rr)
    assert np.array_equal(bins.ids.cpu().numpy().view(np.uint32).astype(np.int64), ii.astype(np.int64))
    assert np.array_equal(bins.keys.cpu().numpy().view(np.uint64), kk)


@pytest.mark.parametrize("n", [3000, 40000])
def test_binning_equal_depths_bit_exact(n):
    """Gaussians on the plane z = 3 seen head-on: every depth is the same
    float, so each tile's order is by slot alone and the sort meets runs of
    thousands of equal keys (tiles above and below the on-chip size)."""
    import time
    sc = synth.uniform_box_scene(7, n, lo=(-1.0, -1.0, 3.0), hi=(1.0, 1.0, 3.0), log_scale_mu=-3.5)
    vw = _eye_view(n, 256, 256, 100.0, 128.0, 128.0)
    ref, r = _records_from_oracle(sc, vw)[0]
    assert np.all(r[ref["radius"] > 0, 14] == np.float32(3.0))
    tile = (16, 16)
    rr, kk, ii = O.bin_view(r[:, 0], r[:, 1], ref["radius"], r[:, 14], 256, 256, *tile, ext=r[:, 2:4])
    counts = rr[:, 1] - rr[:, 0]
    proj = torch.as_tensor(r).cuda()
    views = _lib.Views.from_synth(vw)
    cfg = _lib.config(tile=tile)
    bins = _lib.Bins(views.num_tiles(cfg), len(ii))
    status = _lib.new_status()
    _lib.gs_bin_sort(views, cfg, proj, bins, status)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _lib.gs_bin_sort(views, cfg, proj, bins, status)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert status[0].item() == 0 and bins.counters[0].item() == len(ii)
    assert np.array_equal(bins.tile_ranges.cpu().numpy().reshape(-1, 2).astype(np.int64), rr)
    assert np.array_equal(bins.ids.cpu().numpy().view(np.uint32).astype(np.int64), ii.astype(np.int64))
    assert np.array_equal(bins.keys.cpu().numpy().view(np.uint64), kk)
    print(f"equal depths: {len(ii)} instances, largest tile {counts.max()}, bin+sort {dt * 1e3:.2f} ms")
    assert dt < 2.0   # a sanity bound only


def _large_tile_records(kind):
    """Projected records with crowded tiles. "fallback": a 64x48 view (12
    tiles of 16x16) with one tile of > 60000 instances, more runs than the
    view's run list (2 per tile) holds, so one block sorts it whole
    (partition, then runs and the chunk-and-merge path). "split": a 256x192
    view (192 tiles) with three tiles of ~7000 instances whose runs all fit
    the list and are sorted by any block."""
    if kind == "fallback":
        rng, n, W, H, spots, per, side = np.random.default_rng(11), 80000, 64, 48, ((17, 17),), 60000, 13
    else:
        rng, n, W, H, spots, per, side = (np.random.default_rng(12), 40000, 256, 192,
                                          ((36, 36), (164, 100), (100, 148)), 7000, 8)
    r = np.zeros((n, 16), np.float32)
    r[:, 0] = rng.uniform(0, W, n)
    r[:, 1] = rng.uniform(0, H, n)
    r[:, 11] = rng.integers(1, 3, n)
    r[:, 14] = rng.uniform(1.0, 9.0, n).astype(np.float32)
    r[:, 2] = r[:, 11] * rng.uniform(0.3, 1.0, n)
    r[:, 3] = r[:, 11]
    for c, (x0, y0) in enumerate(spots):
        sl = slice(c * per, (c + 1) * per)
        r[sl, 0] = rng.uniform(x0, x0 + side, per)
        r[sl, 1] = rng.uniform(y0, y0 + side, per)
    return r, W, H


@pytest.mark.parametrize("kind", ["split", "fallback"])
def test_binning_large_tiles_bit_exact(kind):
    """Tiles of > 4096 instances: split into runs of depth bins sorted by
    any block, or (too many runs for the list) sorted whole by one block.
    The result must still equal the oracle's."""
    r, W, H = _large_tile_records(kind)
    n = r.shape[0]
    vw = synth.Views(np.zeros((1, 12), np.float32), np.ones((1, 4), np.float32), np.array([W], np.int32),
                     np.array([H], np.int32), np.array([0]), np.array([n]))
    views = _lib.Views.from_synth(vw)
    cfg = _lib.config(tile=(16, 16))
    rr, kk, ii = O.bin_view(r[:, 0], r[:, 1], r[:, 11].astype(np.int32), r[:, 14], W, H, 16, 16, ext=r[:, 2:4])
    counts = rr[:, 1] - rr[:, 0]
    T = len(counts)
    if kind == "split":
        assert (counts > 4096).sum() == 3 and counts.max() < 2 * 4096   # at most ~8 runs each: 24 <= T
    else:
        assert counts.max() > 16384 and -(-counts.max() // 2048) > 2 * T   # at least 30 runs: more than 2T
    bins = _lib.Bins(views.num_tiles(cfg), len(ii))
    status = _lib.new_status()
    _lib.gs_bin_sort(views, cfg, torch.as_tensor(r).cuda(), bins, status)
    torch.cuda.synchronize()
    assert status[0].item() == 0
    assert np.array_equal(bins.tile_ranges.cpu().numpy().reshape(-1, 2), rr)
    assert np.array_equal(bins.keys.cpu().numpy().view(np.uint64), kk)
    assert np.array_equal(bins.ids.cpu().numpy().view(np.uint32).astype(np.int64), ii)


def test_binning_split_tiles_across_views_bit_exact():
    """Two views with crowded tiles in one call: the split tiles of both views
    share the run list and the sort's queue; each view's lists must equal the
    oracle's (slots offset by the view's slot base)."""
    ra, W, H = _large_tile_records("split")
    rb, _, _ = _large_tile_records("split")
    rb = rb.copy()
    rb[:, 0] = W - rb[:, 0]          # mirrored: crowded tiles elsewhere in the second view
    rb[:, 14] = rb[:, 14][::-1]      # other depths
    na, nb = ra.shape[0], rb.shape[0]
    vw = synth.Views(np.zeros((2, 12), np.float32), np.ones((2, 4), np.float32), np.array([W, W], np.int32),
                     np.array([H, H], np.int32), np.array([0, na]), np.array([na, nb]))
    views = _lib.Views.from_synth(vw)
    cfg = _lib.config(tile=(16, 16))
    refs = [O.bin_view(r[:, 0], r[:, 1], r[:, 11].astype(np.int32), r[:, 14], W, H, 16, 16, ext=r[:, 2:4])
            for r in (ra, rb)]
    assert all((rr[:, 1] - rr[:, 0]).max() > 4096 for rr, _, _ in refs)
    n_inst = sum(len(ii) for _, _, ii in refs)
    bins = _lib.Bins(views.num_tiles(cfg), n_inst)
    status = _lib.new_status()
    _lib.gs_bin_sort(views, cfg, torch.as_tensor(np.concatenate([ra, rb])).cuda(), bins, status)
    torch.cuda.synchronize()
    assert status[0].item() == 0 and bins.counters[0].item() == n_inst
    ranges = bins.tile_ranges.cpu().numpy().reshape(-1, 2).astype(np.int64)
    keys = bins.keys.cpu().numpy().view(np.uint64)
    ids = bins.ids.cpu().numpy().view(np.uint32).astype(np.int64)
    base = 0
    for v, (rr, kk, ii) in enumerate(refs):
        tb, sb = views.tile_base(cfg, v), views.slot_base(v)
        assert np.array_equal(ranges[tb:tb + rr.shape[0]] - base, rr)
        sl = slice(base, base + len(ii))
        assert np.array_equal(ids[sl] - sb, ii.astype(np.int64))
        assert np.array_equal(keys[sl], (kk & np.uint64(0xffffffff00000000)) | ((kk & np.uint64(0xffffffff)) +
                                                                              np.uint64(sb)))
        base += len(ii)


# ---------------------------------------------------------------------------
# rendering
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", list(CASES))
def test_render_parity(case):
    sc, vw = CASES[case]()
    bg = (0.1, 0.2, 0.3)
    _, _, _, image, _ = gpu_forward(sc, vw, bg=bg)
    ref = oracle_forward(sc, vw, bg=bg)
    err, flagged = image_errors(split(image, vw), ref)
    assert err <= 1e-4, (err, flagged)
    assert flagged <= 0.01 * vw.pixels


def test_render_edge_cases():
    # nothing visible: every Gaussian behind the camera -> background only
    sc = synth.uniform_box_scene(0, 100, lo=(-1, -1, -3), hi=(1, 1, -1))
    vw = _eye_view(100, 37, 23, 40.0)
    _, _, _, image, _ = gpu_forward(sc, vw, bg=(0.25, 0.5, 0.75))
    img = split(image, vw)[0]
    assert np.array_equal(img, np.broadcast_to(np.array([0.25, 0.5, 0.75], np.float32)[:, None, None], img.shape))
    # a 1x1 image and a non-finite Gaussian
    sc = synth.uniform_box_scene(1, 30, lo=(-0.1, -0.1, 2), hi=(0.1, 0.1, 3))
    sc.means[3, 1] = np.inf
    vw = _eye_view(30, 1, 1, 20.0)
    _, _, _, image, proj = gpu_forward(sc, vw)
    ref = oracle_forward(sc, vw)
    err, _ = image_errors(split(image, vw), ref)
    assert err <= 1e-4
    assert proj[3, 11].item() == 0.0


def test_batched_views_bit_equal_single_views():
    sc, vw = CASES["orbit_4views"]()
    _, _, _, image, _ = gpu_forward(sc, vw)
    imgs = split(image, vw)
    for v in range(vw.n):
        one = vw.select([v])
        _, _, _, im1, _ = gpu_forward(sc, one)
        assert np.array_equal(split(im1, one)[0], imgs[v])


def test_permutation_invariance_bit_exact():
    sc, vw = _reduced_c2(n=8000, W=160, H=100)
    # keep Gaussians of distinct float32 camera depth (camera at z=-6, R=I)
    cz = (sc.means[:, 2].astype(np.float64) + 6.0).astype(np.float32)
    _, first = np.unique(cz, return_index=True)
    sc = sc.subset(np.sort(first))
    vw = synth._views(synth.look_at((0.0, 0.0, -6.0)), 1000.0 * 160 / 1237.0, 160, 100, 0, sc.n)
    _, _, _, a, _ = gpu_forward(sc, vw)
    perm = np.random.default_rng(3).permutation(sc.n)
    _, _, _, b, _ = gpu_forward(sc.permuted(perm), vw)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_tile_size_invariance_bit_exact():
    sc, vw = _reduced_c2(n=8000, W=170, H=90)
    imgs = [gpu_forward(sc, vw, tile=t)[3].cpu().numpy() for t in [(16, 16), (8, 8), (16, 8), (32, 8), (32, 16), (32, 32)]]
    for im in imgs[1:]:
        assert np.array_equal(imgs[0], im)


# ---------------------------------------------------------------------------
# backward
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", list(CASES))
def test_backward_parity(case):
    _backward_parity(*CASES[case]())


@pytest.mark.parametrize("deg", [0, 1, 2])
def test_backward_parity_several_views_low_degree(deg):
    """The several-view projection backward at SH degrees 0-2 (the SH
    gradients leave one float per store for degrees 0 and 2, 16 bytes per
    store for degree 1): 4 orbit views of a clustered scene."""
    sc = synth.cluster_scene(5, 20000, sh_degree=deg)
    vw = synth._views(synth.orbit_viewmats(4), 1000.0 * 200 / 979.0, 200, 112, 0, sc.n)
    _backward_parity(sc, vw)


def _backward_parity(sc, vw):
    bg = (0.3, 0.1, 0.2)
    rast, g, views, image, proj = gpu_forward(sc, vw, bg=bg)
    ref = oracle_forward(sc, vw, bg=bg)
    ups = upstream(vw, ref)
    up = torch.as_tensor(np.concatenate([u.reshape(-1) for u in ups])).cuda()
    grads, dvm, dtw = rast.backward(g, views, proj, image, up)
    torch.cuda.synchronize()
    rg, dRt, tw, g2ds = O.backward(sc, vw, ref, [u.astype(np.float64) for u in ups], params=O.Params(bg=bg))
    # per-slot 2D gradients first (most diagnostic)
    G2 = grads.grad2d.cpu().numpy()
    for v in range(vw.n):
        sb = views.slot_base(v)
        got = G2[sb: sb + int(vw.gauss_count[v])][:, :9]
        check_grad(got, conic_to_cov_grads(g2ds[v], ref[v]["proj"]["conic"]), f"grad2d view {v}")
    for name in ["means", "log_scales", "quats", "opacity_logits", "sh"]:
        check_grad(getattr(grads, name).cpu().numpy(), rg[name], name)
    check_grad(dvm.cpu().numpy(), dRt, "dL/d(R,t)")
    check_grad(dtw.cpu().numpy(), tw, "twist")


def test_maximum_view_count_parity():
    """GS_MAX_VIEWS (64) views of one scene in one call: images, mean and
    pose gradients against the oracle."""
    sc, vw = synth.orbit_views(0, 3000, 64, 48, 32, 1000.0 * 48 / 979.0)
    assert vw.n == _lib.GS_MAX_VIEWS
    bg = (0.2, 0.1, 0.3)
    rast, g, views, image, proj = gpu_forward(sc, vw, bg=bg)
    ref = oracle_forward(sc, vw, bg=bg)
    err, flagged = image_errors(split(image, vw), ref)
    assert err <= 1e-4, (err, flagged)
    assert flagged <= 0.01 * vw.pixels
    ups = upstream(vw, ref)
    up = torch.as_tensor(np.concatenate([u.reshape(-1) for u in ups])).cuda()
    grads, dvm, dtw = rast.backward(g, views, proj, image, up)
    torch.cuda.synchronize()
    rg, dRt, tw, _ = O.backward(sc, vw, ref, [u.astype(np.float64) for u in ups], params=O.Params(bg=bg))
    check_grad(grads.means.cpu().numpy(), rg["means"], "means, 64 views")
    check_grad(dvm.cpu().numpy(), dRt, "dL/d(R,t), 64 views")
    check_grad(dtw.cpu().numpy(), tw, "twist, 64 views")


@pytest.mark.parametrize("case", ["orbit_4views", "uneven_3scenes"])
def test_multiview_projection_backward_adds_views_in_order(case):
    """The several-view projection backward (per block, chains over per-view
    lists or by owner lanes) adds a Gaussian's views in ascending order: two
    calls agree bit for bit, and the mean and SH-coefficient gradients match
    one-view calls that accumulate the views in ascending order into zeroed
    buffers (each view's term computed by the one-view kernel)."""
    sc, vw = CASES[case]()
    rast, g, views, image, proj = gpu_forward(sc, vw)
    up = torch.randn(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    n_slots = int(np.sum(vw.gauss_count))
    grad2d = torch.empty(max(1, n_slots), _lib.GS_GRAD2D_FLOATS, device="cuda")
    status = _lib.new_status()
    _lib.gs_rasterize_bwd(views, rast.cfg, proj, rast.bins, image, up, grad2d, status)
    outs = []
    for _ in range(2):
        gr = _lib.Grads(g.n, g.sh_degree, n_slots, vw.n)
        gr.grad2d = grad2d
        for t in (gr.means, gr.log_scales, gr.quats, gr.opacity_logits, gr.sh, gr.pose_partials):
            t.fill_(float("nan"))
        _lib.gs_project_bwd(g, views, rast.cfg, proj, gr, True, status)
        torch.cuda.synchronize()
        assert int(status[0].item()) == 0
        outs.append([t.cpu().numpy() for t in (gr.means, gr.log_scales, gr.quats, gr.opacity_logits, gr.sh,
                                               gr.pose_partials)])
    for a, b in zip(*outs):
        assert not np.isnan(a).any() and np.array_equal(a.view(np.uint32), b.view(np.uint32))
    # the views one by one, accumulating
    acc = _lib.Grads(g.n, g.sh_degree, n_slots, vw.n)
    for t in (acc.means, acc.log_scales, acc.quats, acc.opacity_logits, acc.sh):
        t.zero_()
    cfg_acc = _lib.config(tile=rast.tile, accumulate_grads=True)
    for v in range(vw.n):
        vv = _lib.Views(views.viewmats[v:v + 1], views.intrinsics[v:v + 1], views.width[v:v + 1],
                        views.height[v:v + 1], views.gauss_begin[v:v + 1], views.gauss_count[v:v + 1])
        sb, cnt = views.slot_base(v), int(vw.gauss_count[v])
        one = _lib.Grads(g.n, g.sh_degree, cnt, 1)
        for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            setattr(one, name, getattr(acc, name))
        one.grad2d = grad2d[sb:sb + cnt]
        _lib.gs_project_bwd(g, vv, cfg_acc, proj[sb:sb + cnt], one, True, status)
    torch.cuda.synchronize()
    assert int(status[0].item()) == 0
    for got, ref in ((outs[0][0], acc.means.cpu().numpy()), (outs[0][4], acc.sh.cpu().numpy())):
        assert np.allclose(got, ref, rtol=1e-6, atol=1e-6 * np.abs(ref).max())
        assert np.array_equal(got == 0, ref == 0)


def test_pose_only_backward_matches_full():
    sc, vw = CASES["orbit_4views"]()
    rast, g, views, image, proj = gpu_forward(sc, vw)
    up = torch.randn(views.num_image_floats(), device="cuda")
    _, dvm_full, _ = rast.backward(g, views, proj, image, up, want_gaussian_grads=True)
    dvm_full = dvm_full.clone()
    _, dvm_pose, _ = rast.backward(g, views, proj, image, up, want_gaussian_grads=False)
    torch.cuda.synchronize()
    check_grad(dvm_pose.cpu().numpy(), dvm_full.cpu().numpy(), "pose-only", rel_norm=1e-5, rel_elem=1e-5,
               abs_frac=1e-6)


def test_autograd_and_pose_residual_chain():
    """images -> L = <w, images>; gradients of the 6D/translation pose
    residuals (away from the identity) through torch match the oracle's
    dL/d(R', t') chained through the FP64 pose-residual oracle."""
    import dataclasses

    from oracle import pose as OP
    from paper_2509_25191_gb300 import pose
    from paper_2509_25191_gb300.autograd import RasterizeViews
    sc, vw = CASES["orbit_4views"]()
    rng = np.random.default_rng(21)
    dr0 = (OP.identity_6d(vw.n) + 0.02 * rng.standard_normal((vw.n, 6))).astype(np.float32)
    dt0 = (0.01 * rng.standard_normal((vw.n, 3))).astype(np.float32)
    base = torch.as_tensor(vw.viewmats).cuda()
    dr = torch.as_tensor(dr0).cuda().requires_grad_(True)
    dt = torch.as_tensor(dt0).cuda().requires_grad_(True)
    g = _lib.Gaussians.from_scene(sc)
    params = [t.clone().requires_grad_(True) for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh)]
    vm = pose.apply_residual(base, dr, dt)
    # the oracle renders at the refined poses the GPU used (float32)
    vw_ref = dataclasses.replace(vw, viewmats=vm.detach().cpu().numpy().astype(np.float32))
    assert np.allclose(vw_ref.viewmats, OP.apply_residual(vw.viewmats, dr0, dt0), atol=1e-5)
    ref = oracle_forward(sc, vw_ref)
    ups = upstream(vw_ref, ref, seed=5)
    w = torch.as_tensor(np.concatenate([u.reshape(-1) for u in ups])).cuda()
    layout = (vw.width, vw.height, vw.gauss_begin, vw.gauss_count)
    img = RasterizeViews.apply(*params, vm, torch.as_tensor(vw.intrinsics).cuda(), layout, Rasterizer())
    (img * w).sum().backward()
    rg, dRt, _, _ = O.backward(sc, vw_ref, ref, [u.astype(np.float64) for u in ups])
    d_dr, d_dt = OP.residual_vjp(vw.viewmats, dr0, dt0, dRt)
    check_grad(dr.grad.cpu().numpy(), d_dr, "d(6D residual)")
    check_grad(dt.grad.cpu().numpy(), d_dt, "d(translation residual)")
    check_grad(params[0].grad.cpu().numpy(), rg["means"], "means via autograd")


def test_autograd_shared_rasterizer_two_forwards():
    """Two forwards through one Rasterizer (different views), then one
    backward of both: each backward uses its own forward's tile lists, so the
    gradients equal those of two separate rasterizers."""
    from paper_2509_25191_gb300.autograd import RasterizeViews
    sc, vw = CASES["orbit_4views"]()
    g = _lib.Gaussians.from_scene(sc)
    parts = [vw.select([0, 1]), vw.select([2, 3])]
    gen = torch.Generator("cuda").manual_seed(9)
    ws = [torch.randn(3 * int((p.width * p.height).sum()), device="cuda", generator=gen) for p in parts]

    def run(shared):
        params = [t.clone().requires_grad_(True) for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh)]
        rast = Rasterizer()
        loss = 0.0
        for p, w in zip(parts, ws):
            layout = (p.width, p.height, p.gauss_begin, p.gauss_count)
            img = RasterizeViews.apply(*params, torch.as_tensor(p.viewmats).cuda(),
                                       torch.as_tensor(p.intrinsics).cuda(), layout,
                                       rast if shared else Rasterizer())
            loss = loss + (img * w).sum()
        loss.backward()
        return [t.grad.cpu().numpy() for t in params]

    shared, separate = run(True), run(False)
    for name, a, b in zip(("means", "log_scales", "quats", "opacity", "sh"), shared, separate):
        check_grad(a, b, f"shared rasterizer {name}", 1e-4, 1e-3, 1e-6)


def test_l1_loss_kernel():
    a = torch.rand(3 * 37 * 41 + 3, device="cuda")
    b = torch.rand_like(a)
    b[5] = a[5]
    loss = torch.empty(1, device="cuda")
    grad = torch.empty_like(a)
    _lib.gs_l1_loss(a, b, loss, grad)
    torch.cuda.synchronize()
    d = (a - b).double().cpu().numpy()
    assert abs(loss.item() - np.abs(d).mean()) < 1e-6
    assert np.array_equal(grad.cpu().numpy(), (np.sign(d) / d.size).astype(np.float32))


@pytest.mark.parametrize("case", ["small_2k", "clustered_sh3", "orbit_4views", "uneven_3scenes"])
def test_raster_backward_with_the_l1_loss_folded_in(case):
    """gs_rasterize_bwd_l1 forms the mean L1 loss's gradient in the raster
    backward: its 2D gradients equal gs_l1_loss followed by gs_rasterize_bwd
    up to the order of float atomics, and its loss the mean absolute
    difference (some image values equal to the target: zero gradient)."""
    sc, vw = CASES[case]()
    rast, g, views, image, proj = gpu_forward(sc, vw)
    target = torch.rand(image.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(11))
    target[::7] = image[::7]
    n_slots = max(1, views.num_slots())
    loss_a, loss_b = torch.empty(1, device="cuda"), torch.empty(1, device="cuda")
    dimg = torch.empty_like(image)
    a = torch.empty(n_slots, _lib.GS_GRAD2D_FLOATS, device="cuda")
    b = torch.empty_like(a)
    _lib.gs_l1_loss(image, target, loss_a, dimg)
    _lib.gs_rasterize_bwd(views, rast.cfg, proj, rast.bins, image, dimg, a)
    _lib.gs_rasterize_bwd_l1(views, rast.cfg, proj, rast.bins, image, target, loss_b, b)
    torch.cuda.synchronize()
    d = (image - target).double().cpu().numpy()
    assert abs(loss_b.item() - np.abs(d).mean()) <= 1e-6 * max(1.0, np.abs(d).mean())
    assert abs(loss_b.item() - loss_a.item()) <= 1e-6 * loss_a.item()
    A, B = a.cpu().numpy(), b.cpu().numpy()
    assert np.abs(A).max() > 0
    assert np.linalg.norm(B - A) <= 1e-5 * np.linalg.norm(A)
    assert np.abs(B - A).max() <= 1e-5 * np.abs(A).max()


def test_bounded_wait_runs_out_and_reports():
    """The projection kernels' bounded wait, on a copy barrier that nothing
    completes, gives up after about a second and reports GS_ERR_TIMEOUT in
    the status word; nothing faults and the context keeps running kernels."""
    import time
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t = time.perf_counter()
    _lib.gs_check_bounded_wait(status)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    assert status.tolist() == [_lib.GS_ERR_TIMEOUT, 0, 0, 0]
    assert 0.5 < dt < 30.0, dt
    assert "bounded wait" in _lib.error_string(_lib.GS_ERR_TIMEOUT)
    # the context still runs the library's kernels
    a = torch.zeros(3 * 64, device="cuda")
    b = torch.full_like(a, 0.5)
    loss = torch.empty(1, device="cuda")
    _lib.gs_l1_loss(a, b, loss, torch.empty_like(a))
    torch.cuda.synchronize()
    assert loss.item() == 0.5


# ---------------------------------------------------------------------------
# CUDA graph capture of a whole step
# ---------------------------------------------------------------------------

def test_graph_step_input_slots():
    """A two-slot GraphStep captures one graph per input slot (target, view
    matrices and Gaussian parameters) over shared buffers, with the loss and
    pose gradient kept per slot; replaying a slot gives the results of a
    single-slot step built on that slot's inputs, and leaves the other
    slot's results as they were."""
    from paper_2509_25191_gb300.step import GraphStep
    sc, vw = CASES["clustered_sh3"]()
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    gen = torch.Generator("cuda").manual_seed(3)
    t0 = torch.rand(views.num_image_floats(), device="cuda", generator=gen)
    t1 = torch.rand(views.num_image_floats(), device="cuda", generator=gen)
    vm1 = views.viewmats.clone()
    vm1[:, 9:] += 0.02
    # slot 1's Gaussians: slightly more opaque and moved
    g1 = _lib.Gaussians(g.means + 0.01 * torch.randn(g.means.shape, device="cuda", generator=gen),
                        g.log_scales.clone(), g.quats.clone(), g.opacity_logits + 0.25, g.sh.clone())
    step = GraphStep(g, views, t0, slots=2, slot_gaussians=True)
    step.target_slots[1].copy_(t1)
    step.viewmat_slots[1].copy_(vm1)
    for dst, src in zip(_gauss_tensors(step.gauss_slots[1]), _gauss_tensors(g1)):
        dst.copy_(src)
    got = []
    for sl in (0, 1, 0):
        step.replay(sl)
        got.append((step.loss_slots[sl].clone(), step.dviewmat_slots[sl].clone(), step.image.clone(),
                    step.grads.means.clone(), step.grads.opacity_logits.clone()))
    # slot 1's results survive the last replay of slot 0
    assert torch.equal(step.loss_slots[1], got[1][0]) and torch.equal(step.dviewmat_slots[1], got[1][1])
    views1 = _lib.Views(vm1, views.intrinsics, views.width, views.height, views.gauss_begin, views.gauss_count)
    refs = []
    for gg, vv, tt in ((g, views, t0), (g1, views1, t1)):
        ref = GraphStep(gg, vv, tt)
        ref.replay()
        refs.append((ref.loss.clone(), ref.dviewmat.clone(), ref.image.clone(), ref.grads.means.clone(),
                     ref.grads.opacity_logits.clone()))
    torch.cuda.synchronize()
    assert not step.check()
    for (l, d, im, gm, go), (rl, rd, rim, rgm, rgo) in zip(got, [refs[0], refs[1], refs[0]]):
        assert torch.equal(im, rim)
        assert abs(float(l) - float(rl)) <= 1e-6 * abs(float(rl))
        check_grad(d.cpu().numpy(), rd.cpu().numpy(), "slot pose gradient", 1e-4, 1e-4, 1e-6)
        check_grad(gm.cpu().numpy(), rgm.cpu().numpy(), "slot mean gradient", 1e-3, 1e-3, 1e-6)
        check_grad(go.cpu().numpy(), rgo.cpu().numpy(), "slot opacity gradient", 1e-3, 1e-3, 1e-6)
    assert not torch.equal(got[0][2], got[1][2])


def _gauss_tensors(g):
    return (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh)


def test_graph_capture_replays_step():
    sc, vw = CASES["orbit_4views"]()
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    rast = Rasterizer()
    image0, proj0 = rast.forward(g, views)
    up = torch.randn(views.num_image_floats(), device="cuda")
    grads0, dvm0, _ = rast.backward(g, views, proj0, image0, up)
    ref_img, ref_gm, ref_dvm = image0.clone(), grads0.means.clone(), dvm0.clone()
    torch.cuda.synchronize()
    rast.reserve(views, int(rast.last_instances * 1.5) + 1024)
    proj = torch.empty_like(proj0)
    image = torch.empty_like(image0)
    grads = rast.grads_buffers(g, views)
    dvm = torch.empty(vw.n, 12, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            rast.project(g, views, proj)
            bins = rast.bin_sort(views, proj)
            rast.render(views, proj, bins, image)
            _lib.gs_render_bwd(g, views, rast.cfg, proj, bins, image, up, grads, True, rast.status)
            _lib.gs_pose_grad(views, grads.pose_partials, grads.n_blocks, dvm)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    rast.check_status()
    assert torch.equal(image, ref_img)
    check_grad(grads.means.cpu().numpy(), ref_gm.cpu().numpy(), "graph means", 1e-5, 1e-4, 1e-6)
    check_grad(dvm.cpu().numpy(), ref_dvm.cpu().numpy(), "graph pose", 1e-5, 1e-4, 1e-6)
