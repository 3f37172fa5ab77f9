"""The boundary's caller-facing contracts on the GPU, through the C ABI:
gradient accumulation (+=), the per-pixel last-contributor record, the
one-buffer workspace, the status read, and re-planning of a captured step
after a capacity overflow."""
import numpy as np
import pytest
import torch

from paper_2509_25191_gb300 import _lib
from paper_2509_25191_gb300.autograd import Rasterizer
from paper_2509_25191_gb300.step import GraphStep
from tests.gpu_util import gpu_forward, split
from tests.test_gpu_parity import CASES

pytestmark = pytest.mark.gpu

GRAD_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _grads_of(gr):
    return [getattr(gr, n).cpu().numpy().copy() for n in GRAD_NAMES]


@pytest.mark.parametrize("use_tma", [True, False])
@pytest.mark.parametrize("case", ["clustered_sh3", "subset_view", "uneven_3scenes"])
def test_accumulated_projection_backward_is_twice_the_single(case, use_tma):
    """Two accumulating calls on the same 2D gradients into zeroed buffers
    give exactly twice one overwriting call (each call adds one total per
    value, summed over the views first: x + x = 2x in float32), whatever
    the tensor-copy setting; Gaussians no view sees keep the value the
    caller put there."""
    sc, vw = CASES[case]()
    rast, g, views, image, proj = gpu_forward(sc, vw)
    up = torch.randn(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    n_slots = views.num_slots()
    grad2d = torch.empty(max(1, n_slots), _lib.GS_GRAD2D_FLOATS, device="cuda")
    status = _lib.new_status()
    _lib.gs_rasterize_bwd(views, rast.cfg, proj, rast.bins, image, up, grad2d, status)
    one = _lib.Grads(g.n, g.sh_degree, n_slots, views.n)
    one.grad2d = grad2d
    _lib.gs_project_bwd(g, views, _lib.config(tile=rast.tile, use_tma=use_tma), proj, one, True, status)
    acc = _lib.Grads(g.n, g.sh_degree, n_slots, views.n)
    acc.grad2d = grad2d
    sentinel = 0.25
    for n in GRAD_NAMES:
        getattr(acc, n).zero_()
    covered = np.zeros(g.n, bool)
    for b, c in zip(vw.gauss_begin, vw.gauss_count):
        covered[b:b + c] = True
    unseen = torch.as_tensor(~covered, device="cuda")
    for n in GRAD_NAMES:
        getattr(acc, n)[unseen] = sentinel
    cfg_acc = _lib.config(tile=rast.tile, use_tma=use_tma, accumulate_grads=True)
    _lib.gs_project_bwd(g, views, cfg_acc, proj, acc, True, status)
    _lib.gs_project_bwd(g, views, cfg_acc, proj, acc, True, status)
    torch.cuda.synchronize()
    assert int(status[0].item()) == 0
    for name, a, o in zip(GRAD_NAMES, _grads_of(acc), _grads_of(one)):
        a = a.reshape(g.n, -1)
        o = o.reshape(g.n, -1)
        assert np.array_equal(a[covered], 2.0 * o[covered]), name
        assert np.all(a[~covered] == sentinel), name


@pytest.mark.parametrize("case", ["clustered_sh3", "subset_view"])
def test_one_view_projection_backward_is_deterministic(case):
    """A one-view projection backward runs the chain only over the Gaussians
    with a nonzero 2D gradient, compacted per block in an order fixed by
    their indices: two calls give bitwise the same parameter gradients and
    pose partials, and the Gaussians without a gradient (or outside the
    view's range) get exact zeros."""
    sc, vw = CASES[case]()
    assert vw.n == 1
    rast, g, views, image, proj = gpu_forward(sc, vw)
    up = torch.randn(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    n_slots = views.num_slots()
    grad2d = torch.empty(max(1, n_slots), _lib.GS_GRAD2D_FLOATS, device="cuda")
    status = _lib.new_status()
    _lib.gs_rasterize_bwd(views, rast.cfg, proj, rast.bins, image, up, grad2d, status)
    runs = []
    for _ in range(2):
        gr = _lib.Grads(g.n, g.sh_degree, n_slots, views.n)
        gr.grad2d = grad2d
        for n in GRAD_NAMES:
            getattr(gr, n).fill_(7.0)   # every value must be written
        _lib.gs_project_bwd(g, views, rast.cfg, proj, gr, True, status)
        torch.cuda.synchronize()
        runs.append(_grads_of(gr) + [gr.pose_partials.cpu().numpy().copy()])
    assert int(status[0].item()) == 0
    for a, b in zip(runs[0], runs[1]):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    g2 = grad2d.cpu().numpy()[:, :9]
    active = np.zeros(g.n, bool)
    b0, c0 = int(vw.gauss_begin[0]), int(vw.gauss_count[0])
    active[b0:b0 + c0] = np.any(g2[:c0] != 0, axis=1)
    assert 0 < active.sum() < g.n
    for a in runs[0][:5]:
        assert np.all(a.reshape(g.n, -1)[~active] == 0.0)


def test_accumulated_render_backward_adds_across_calls():
    """gs_render_bwd (raster + projection backward) twice with accumulation
    gives twice one call, up to the last bits of the raster backward's float
    atomics."""
    sc, vw = CASES["orbit_4views"]()
    rast, g, views, image, proj = gpu_forward(sc, vw)
    up = torch.randn(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    one = _lib.Grads(g.n, g.sh_degree, views.num_slots(), views.n)
    _lib.gs_render_bwd(g, views, rast.cfg, proj, rast.bins, image, up, one)
    acc = _lib.Grads(g.n, g.sh_degree, views.num_slots(), views.n)
    for n in GRAD_NAMES:
        getattr(acc, n).zero_()
    cfg_acc = _lib.config(tile=rast.tile, accumulate_grads=True)
    _lib.gs_render_bwd(g, views, cfg_acc, proj, rast.bins, image, up, acc)
    _lib.gs_render_bwd(g, views, cfg_acc, proj, rast.bins, image, up, acc)
    torch.cuda.synchronize()
    for name, a, o in zip(GRAD_NAMES, _grads_of(acc), _grads_of(one)):
        assert np.linalg.norm(a - 2 * o) <= 1e-5 * np.linalg.norm(2 * o), name


@pytest.mark.parametrize("tile", [(16, 16), (32, 16), (8, 8)])
@pytest.mark.parametrize("case", ["small_2k", "clustered_sh3", "orbit_4views", "uneven_3scenes"])
def test_last_contributor_replay_equals_full_replay(case, tile):
    """The backward that ends each pixel at its last composited Gaussian
    gives the 2D gradients of the replay to saturation (up to float-atomic
    order), evaluates no more pairs, and every recorded end lies inside its
    tile's range."""
    sc, vw = CASES[case]()
    rast, g, views, image, proj = gpu_forward(sc, vw, tile=tile)
    assert rast.bins.last_contrib is not None
    up = torch.randn(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    n_slots = max(1, views.num_slots())
    cfg = _lib.config(tile=tile, count_pairs=True)
    a = torch.empty(n_slots, _lib.GS_GRAD2D_FLOATS, device="cuda")
    b = torch.empty_like(a)
    _lib.gs_rasterize_bwd(views, cfg, proj, rast.bins, image, up, a, use_last=True)
    ev_last, co_last = _lib.pair_counts(rast.bins)[2:]
    _lib.gs_rasterize_bwd(views, cfg, proj, rast.bins, image, up, b, use_last=False)
    ev_tot, co_tot = _lib.pair_counts(rast.bins)[2:]      # the counters add up over calls
    ev_full, co_full = ev_tot - ev_last, co_tot - co_last
    torch.cuda.synchronize()
    A, B = a.cpu().numpy(), b.cpu().numpy()
    assert np.linalg.norm(A - B) <= 1e-5 * np.linalg.norm(B) + 1e-30
    assert np.abs(A - B).max() <= 1e-5 * np.abs(B).max() + 1e-30
    assert co_last == co_full and ev_last <= ev_full
    # the recorded ends against the tile ranges
    ranges = rast.bins.tile_ranges.cpu().numpy().reshape(-1, 2)
    last = rast.bins.last_contrib.cpu().numpy()
    off = 0
    tw, th = tile
    for v in range(views.n):
        W, H = int(vw.width[v]), int(vw.height[v])
        Gx = (W + tw - 1) // tw
        yy, xx = np.mgrid[0:H, 0:W]
        t = views.tile_base(cfg, v) + (yy // th) * Gx + xx // tw
        e = last[off:off + W * H].reshape(H, W)
        assert np.all(e >= ranges[t, 0]) and np.all(e <= ranges[t, 1])
        off += W * H


@pytest.mark.parametrize("case", ["clustered_sh3", "orbit_4views", "uneven_3scenes"])
def test_tile_work_record_orders_without_changing_results(case):
    """The kept per-tile work record only orders the raster kernels' tiles:
    whatever it holds (zeros, garbage, the previous forward's lengths) the
    image is bit-identical and the 2D gradients agree up to float-atomic
    order; after a forward it holds each tile's replay length, the largest
    last-contributor offset of its pixels from the tile's start."""
    sc, vw = CASES[case]()
    tile = (16, 16)
    rast, g, views, image, proj = gpu_forward(sc, vw, tile=tile)
    b, cfg = rast.bins, rast.cfg
    T = views.num_tiles(cfg)
    assert b.tile_work is not None and 0 < T < 16 * torch.cuda.get_device_properties(0).multi_processor_count
    up = torch.randn(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(8))
    ref = torch.empty(max(1, views.num_slots()), _lib.GS_GRAD2D_FLOATS, device="cuda")
    _lib.gs_rasterize_bwd(views, cfg, proj, b, image, up, ref)
    R = ref.cpu().numpy()
    gen = torch.Generator("cuda").manual_seed(9)
    for fill in ("zeros", "garbage", "previous"):
        if fill == "zeros":
            b.tile_work.zero_()
        elif fill == "garbage":
            b.tile_work.copy_(torch.randint(-2 ** 31, 2 ** 31 - 1, b.tile_work.shape, generator=gen, device="cuda",
                                            dtype=torch.int64).to(torch.int32))
        img = torch.empty_like(image)
        _lib.gs_render_fwd(views, cfg, proj, b, img, _lib.new_status())
        gd = torch.empty_like(ref)
        _lib.gs_rasterize_bwd(views, cfg, proj, b, img, up, gd)
        torch.cuda.synchronize()
        assert torch.equal(img, image), fill
        D = gd.cpu().numpy()
        assert np.linalg.norm(D - R) <= 1e-5 * np.linalg.norm(R) + 1e-30, fill
    # the record left by the last forward
    work = b.tile_work.cpu().numpy()[:T]
    ranges = b.tile_ranges.cpu().numpy().reshape(-1, 2)
    last = b.last_contrib.cpu().numpy()
    expect = np.zeros(T, np.int64)
    off = 0
    tw, th = tile
    for v in range(views.n):
        W, H = int(vw.width[v]), int(vw.height[v])
        Gx = (W + tw - 1) // tw
        yy, xx = np.mgrid[0:H, 0:W]
        t = (views.tile_base(cfg, v) + (yy // th) * Gx + xx // tw).ravel()
        np.maximum.at(expect, t, last[off:off + W * H].astype(np.int64) - ranges[t, 0])
        off += W * H
    assert np.array_equal(work, expect)


@pytest.mark.parametrize("case", ["clustered_sh3", "orbit_4views"])
def test_overlapped_backward_equals_the_plain_order(case):
    """With gs_config.overlap_prev the raster backward's accumulators and the
    one-view projection backward's gradient rows are zeroed in the tail of
    the kernel ahead (programmatic dependent launches); the backward gives
    the loss, parameter and pose gradients of the plain order, where every
    kernel waits for the work ahead (up to the order of float atomics), on
    a first call and on a second into the same buffers."""
    sc, vw = CASES[case]()
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    target = torch.rand(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(12))
    res = []
    for overlap in (False, True):
        rast = Rasterizer(tile=(16, 16), overlap_prev=overlap)
        image, proj = rast.forward(g, views)
        loss = torch.empty(1, device="cuda")
        out = []
        grads = None
        for _ in range(2):
            grads, dvm, dtw = rast.backward_l1(g, views, proj, image, target, loss, grads=grads)
            torch.cuda.synchronize()
            out.append([loss.cpu().numpy().copy(), dvm.cpu().numpy().copy(), dtw.cpu().numpy().copy()] +
                       _grads_of(grads))
        rast.check_status()
        res.append(out)
    for call in range(2):
        for a, b in zip(res[0][call], res[1][call]):
            assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a) + 1e-30
        # the second call repeats the first
        for a, b in zip(res[1][0], res[1][call]):
            assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a) + 1e-30


def test_workspace_step_equals_the_rasterizer():
    """A forward and backward whose tile lists, 2D gradients and pose
    partials are carved from one caller buffer give the Rasterizer's image
    and gradients."""
    sc, vw = CASES["uneven_3scenes"]()
    rast, g, views, image, proj = gpu_forward(sc, vw)
    up = torch.randn(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(6))
    grads_r, dvm_r, _ = rast.backward(g, views, proj, image, up)
    torch.cuda.synchronize()
    ref = [t.cpu().numpy().copy() for t in (image, dvm_r)] + _grads_of(grads_r)
    cfg = rast.cfg
    cap = int(rast.last_instances) + 100
    size = _lib.gs_workspace_size(views, cfg, g.n, cap)
    ws = torch.empty(size // 4 + 64, dtype=torch.float32, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    cb, g2d_ptr, pp_ptr = _lib.gs_workspace_carve(views, cfg, g.n, cap, base, size)
    lib = _lib.load()
    import ctypes
    status = _lib.new_status()
    st = _lib._stream(None)
    proj2 = torch.empty_like(proj)
    img2 = torch.empty_like(image)
    assert lib.gs_project(ctypes.byref(g.c()), ctypes.byref(views.c()), ctypes.byref(cfg), _lib._ptr(proj2),
                          _lib._ptr(status), st) == 0
    assert lib.gs_bin_sort(ctypes.byref(views.c()), ctypes.byref(cfg), _lib._ptr(proj2), ctypes.byref(cb),
                           _lib._ptr(status), st) == 0
    assert lib.gs_render_fwd(ctypes.byref(views.c()), ctypes.byref(cfg), _lib._ptr(proj2), ctypes.byref(cb),
                             _lib._ptr(img2), _lib._ptr(status), st) == 0
    gr = _lib.Grads(g.n, g.sh_degree, views.num_slots(), views.n)
    cg = gr.c()
    cg.grad2d, cg.pose_partials = g2d_ptr, pp_ptr
    assert lib.gs_render_bwd(ctypes.byref(g.c()), ctypes.byref(views.c()), ctypes.byref(cfg), _lib._ptr(proj2),
                             ctypes.byref(cb), _lib._ptr(img2), _lib._ptr(up), ctypes.byref(cg), 1,
                             _lib._ptr(status), st) == 0
    dvm = torch.empty(views.n, 12, device="cuda")
    assert lib.gs_pose_grad(ctypes.byref(views.c()), ctypes.c_void_p(pp_ptr), gr.n_blocks, _lib._ptr(dvm), None,
                            st) == 0
    assert _lib.gs_status_read(status)[0] == 0
    got = [img2.cpu().numpy(), dvm.cpu().numpy()] + _grads_of(gr)
    assert np.array_equal(got[0], ref[0])                    # the image is deterministic
    for a, b in zip(got[1:], ref[1:]):
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b) + 1e-30


def test_status_read_reports_capacity_overflow():
    sc, vw = CASES["small_2k"]()
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    rast = Rasterizer()
    proj = rast.project(g, views)
    small = _lib.Bins(views.num_tiles(rast.cfg), 10)
    status = _lib.new_status()
    assert _lib.gs_status_read(status) == [0, 0, 0, 0]
    _lib.gs_bin_sort(views, rast.cfg, proj, small, status)
    st = _lib.gs_status_read(status)
    need = int(small.counters[0].item())
    assert st[0] == _lib.GS_ERR_CAPACITY and st[1] == need and st[2] == 0 and need > 10


def test_graph_step_check_recovers_from_an_overflow_once():
    """A captured step planned with too small a capacity reports the
    overflow once, re-plans, and the next replay fits: check() is True once,
    then False, and the image equals that of a step planned from the start."""
    sc, vw = CASES["clustered_sh3"]()
    g = _lib.Gaussians.from_scene(sc)
    views = _lib.Views.from_synth(vw)
    target = torch.rand(views.num_image_floats(), device="cuda", generator=torch.Generator("cuda").manual_seed(7))
    step = GraphStep(g, views, target, tile=(16, 16), capacity=1000)
    step.replay()
    assert step.check() is True
    step.replay()
    assert step.check() is False
    step.replay()
    assert step.check() is False
    ref = GraphStep(g, views, target, tile=(16, 16))
    ref.replay()
    assert ref.check() is False
    torch.cuda.synchronize()
    assert np.array_equal(step.image.cpu().numpy(), ref.image.cpu().numpy())
    assert split(step.image, vw)[0].max() > 0
