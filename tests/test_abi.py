"""The C-ABI library loads and exports every entry point include/gs.h
declares (CPU only: no compute calls)."""
import ctypes
import os
import re


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gs_\w+)\s*\(", src, re.M)))


def test_header_declares_the_rasterizer_entry_points():
    names = _declared()
    for n in ["gs_project", "gs_bin_sort", "gs_render_fwd", "gs_render_bwd", "gs_pose_grad"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2509_25191_gb300 import build as B
    B.build()
    lib = ctypes.CDLL(B.LIB)
    for n in _declared():
        assert hasattr(lib, n), n
    assert lib.gs_version() >= 1
    lib.gs_error_string.restype = ctypes.c_char_p
    assert lib.gs_error_string(3) == b"instance capacity exceeded"
    assert lib.gs_error_string(7) == b"a bounded wait for an asynchronous copy ran out"


def test_host_layout_queries_without_gpu():
    from paper_2509_25191_gb300 import _lib, synth
    sc, vw = synth.uneven_scenes(seeds=(1, 2), sizes=(10, 20), views_per_scene=2,
                                 resolutions=((33, 17), (64, 48)))
    lib = _lib.load()
    cfg = _lib.gs_config()
    lib.gs_config_default(ctypes.byref(cfg))
    assert (cfg.tile_w, cfg.tile_h, cfg.pixel_gate) == (16, 16, 1)
    assert abs(cfg.alpha_min - 1 / 255) < 1e-9 and abs(cfg.alpha_max - 0.99) < 1e-7
    # every field the C default fills, in the binding's layout (the last one
    # tells a shifted layout apart: the C side writes all of them)
    cfg.overlap_prev = 7
    lib.gs_config_default(ctypes.byref(cfg))
    assert (cfg.count_pairs, cfg.accumulate_grads, cfg.use_tma) == (0, 0, 1)
    assert (cfg.fwd_batch, cfg.bwd_batch, cfg.overlap_prev) == (2, 1, 0)
    assert _lib.config(overlap_prev=True).overlap_prev == 1
    views = _lib.Views(None, None, vw.width, vw.height, vw.gauss_begin, vw.gauss_count)
    c = views.c()
    assert lib.gs_num_slots(ctypes.byref(c)) == 60
    assert lib.gs_slot_base(ctypes.byref(c), 3) == 40
    T = sum(((w + 15) // 16) * ((h + 15) // 16) for w, h in zip(vw.width, vw.height))
    assert lib.gs_num_tiles(ctypes.byref(c), ctypes.byref(cfg)) == T
    assert lib.gs_num_image_floats(ctypes.byref(c)) == 3 * int((vw.width * vw.height).sum())


def test_cuda_calls_fail_cleanly_with_bad_arguments():
    """Host-side checks reject bad arguments before touching a device."""
    from paper_2509_25191_gb300 import _lib
    lib = _lib.load()
    assert lib.gs_project(None, None, None, None, None, None) == _lib.GS_ERR_ARG
    assert lib.gs_pose_grad(None, None, 0, None, None, None) == _lib.GS_ERR_ARG
    assert lib.gs_l1_loss(None, None, ctypes.c_int64(-1), None, None, None) == _lib.GS_ERR_ARG
    assert lib.gs_rasterize_bwd_l1(None, None, None, None, None, None, None, None, None, None) == _lib.GS_ERR_ARG


def test_tile_shapes_on_the_host():
    """Every supported tile shape has a tile grid; an unsupported one is
    rejected by the host-side checks before anything is enqueued."""
    from paper_2509_25191_gb300 import _lib, synth
    sc, vw = synth.single_view_small(n=8)
    lib = _lib.load()
    views = _lib.Views(None, None, vw.width, vw.height, vw.gauss_begin, vw.gauss_count)
    c = views.c()
    W, H = int(vw.width[0]), int(vw.height[0])
    for tw, th in [(16, 16), (8, 8), (16, 8), (32, 8), (32, 16), (32, 32)]:
        cfg = _lib.config(tile=(tw, th))
        assert lib.gs_num_tiles(ctypes.byref(c), ctypes.byref(cfg)) == ((W + tw - 1) // tw) * ((H + th - 1) // th)
    bad = _lib.config(tile=(24, 24))
    g = _lib.gs_gaussians()
    assert lib.gs_project(ctypes.byref(g), ctypes.byref(c), ctypes.byref(bad), None, None, None) == \
        _lib.GS_ERR_UNSUPPORTED


def test_host_checks_reject_bad_layouts():
    """Every layout error is caught by the host-side checks and returned
    before anything is enqueued (no device is touched: the pointers below
    are placeholders that are never dereferenced)."""
    import numpy as np
    from paper_2509_25191_gb300 import _lib
    lib = _lib.load()
    fake = ctypes.c_void_p(1 << 20)   # 16-byte aligned, never dereferenced

    def views(widths, heights, begins, counts):
        arrs = (np.asarray(widths, np.int32), np.asarray(heights, np.int32), np.asarray(begins, np.int64),
                np.asarray(counts, np.int64))
        v = _lib.gs_views(len(widths), fake, fake, *(a.ctypes.data for a in arrs))
        return v, arrs

    def project(v, cfg=None, n=100, deg=0):
        g = _lib.gs_gaussians(n, deg, fake, fake, fake, fake, fake)
        cfg = cfg or _lib.config()
        return lib.gs_project(ctypes.byref(g), ctypes.byref(v), ctypes.byref(cfg), fake, None, None)

    ok_v, keep = views([64], [48], [0], [100])
    too_many, k1 = views([8] * 65, [8] * 65, [0] * 65, [10] * 65)
    assert project(too_many) == _lib.GS_ERR_ARG                      # more than GS_MAX_VIEWS views
    zero_w, k2 = views([0], [48], [0], [10])
    assert project(zero_w) == _lib.GS_ERR_ARG                        # empty image
    beyond, k3 = views([64], [48], [90], [20])
    assert project(beyond) == _lib.GS_ERR_ARG                        # view range past the last Gaussian
    overlap, k4 = views([64, 64], [48, 48], [0, 50], [60, 50])
    assert project(overlap) == _lib.GS_ERR_ARG                       # scene ranges overlap
    assert project(ok_v, deg=4) == _lib.GS_ERR_UNSUPPORTED           # SH degree above 3
    bad_alpha = _lib.config()
    bad_alpha.alpha_max = 1.0
    assert project(ok_v, cfg=bad_alpha) == _lib.GS_ERR_ARG           # alpha clamp must be below 1
    assert lib.gs_check_bounded_wait(None, None) == _lib.GS_ERR_ARG


def test_config_defaults_of_the_boundary_flags():
    """Gradients are overwritten unless accumulation is asked for, and the
    projection kernels may use tensor copies unless told not to."""
    from paper_2509_25191_gb300 import _lib
    cfg = _lib.gs_config()
    _lib.load().gs_config_default(ctypes.byref(cfg))
    assert (cfg.accumulate_grads, cfg.use_tma, cfg.count_pairs) == (0, 1, 0)
    c = _lib.config(accumulate_grads=True, use_tma=False)
    assert (c.accumulate_grads, c.use_tma) == (1, 0)


def test_workspace_layout_on_the_host():
    """gs_workspace_size and gs_workspace_carve are host arithmetic: every
    piece is 256-byte aligned, inside the buffer, large enough for its array
    and disjoint from the others (checked on a placeholder address that is
    never dereferenced)."""
    from paper_2509_25191_gb300 import _lib, synth
    sc, vw = synth.uneven_scenes(seeds=(1, 2), sizes=(10, 20), views_per_scene=2,
                                 resolutions=((33, 17), (64, 48)))
    views = _lib.Views(None, None, vw.width, vw.height, vw.gauss_begin, vw.gauss_count)
    cfg = _lib.config(tile=(16, 8))
    n, cap = int(sc.n), 1000
    size = _lib.gs_workspace_size(views, cfg, n, cap)
    base = 1 << 30
    bins, g2d, pp = _lib.gs_workspace_carve(views, cfg, n, cap, base, size)
    T = views.num_tiles(cfg)
    P = views.num_slots()
    blocks = int(_lib.load().gs_pose_blocks(ctypes.c_int64(n)))
    pieces = [(bins.tile_ranges, 8 * T), (bins.keys, 8 * cap), (bins.ids, 4 * cap), (bins.keys_tmp, 8 * cap),
              (bins.tile_order, 4 * T), (bins.tile_scratch, 20 * T), (bins.counters, 4 * _lib.GS_NUM_COUNTERS),
              (bins.last_contrib, 4 * views.pixels), (bins.tile_work, 4 * T), (g2d, 4 * 12 * P),
              (pp, 4 * 12 * views.n * blocks)]
    spans = sorted((p, p + nbytes) for p, nbytes in pieces)
    assert all(p % 256 == 0 and base <= p and e <= base + size for p, e in spans)
    assert all(spans[i][1] <= spans[i + 1][0] for i in range(len(spans) - 1))
    assert bins.capacity == cap
    # too small a buffer, a misaligned one, or bad arguments are rejected
    lib = _lib.load()
    b, gr = _lib.gs_bins(), _lib.gs_grads()
    c = views.c()
    for ws, nbytes in ((base, size - 1), (base + 16, size)):
        assert lib.gs_workspace_carve(ctypes.byref(c), ctypes.byref(cfg), n, cap, ctypes.c_void_p(ws),
                                      ctypes.c_size_t(nbytes), ctypes.byref(b), ctypes.byref(gr)) == _lib.GS_ERR_ARG
    assert _lib.gs_workspace_size(views, cfg, n, -1) == 0
    assert lib.gs_status_read(None, None, None) == _lib.GS_ERR_ARG
