"""GPU parity of the camera global alignment (Section 3.3, Eqs. 2-4) against
the FP64 oracle, through the C ABI: candidate pairs and incidence lists bit
for bit, histogram counts and median order statistics bit for bit, epipolar
distances within a bound derived from float32 arithmetic, loss and camera
gradients at the gradient tolerance, at a small size and at the full
300-camera, 4,096-matches-per-pair size; edge cases; and a property check
that 300 alignment steps reduce the pose error."""
import numpy as np
import pytest
import torch

from oracle import ga as OG
from paper_2509_25191_gb300 import _lib, ga, synth
from tests.gpu_util import check_grad

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _problem(n_views=40, per_pair=700, seed=0, width=1600, height=1066, ragged=True):
    tv, ti, iv, ii = synth.ga_cameras(seed, n_views, width, height)
    pairs = OG.select_pairs(iv, 30.0)
    M = synth.ga_matches(seed, synth.ga_points(seed, 6000), ti, tv, pairs, width, height, per_pair)
    if ragged:       # ragged match counts, two empty pairs
        keep = np.ones(len(M.matches), bool)
        rng = np.random.default_rng(seed + 7)
        offs = [0]
        for m in range(len(pairs)):
            a, b = M.offsets[m], M.offsets[m + 1]
            k = 0 if m in (1, 5) else int(rng.integers(1, b - a + 1))
            keep[a + k:b] = False
            offs.append(offs[-1] + k)
        M = synth.Matches(np.asarray(offs, np.int64), np.ascontiguousarray(M.matches[keep]), M.inlier[keep])
    return tv, ti, iv, ii, pairs, M


def _cuda(*arrs):
    return [torch.as_tensor(np.ascontiguousarray(a)).cuda() for a in arrs]


def _kappa(intr, vms, pairs, offsets, matches):
    """Float32 error scale of each distance: sum_rs |x^'_r| (|E_rs| + |t|)
    |x^_s| / ||l_12|| (FP64, from the inputs)."""
    out = np.zeros(len(matches))
    for m, (i, j) in enumerate(pairs):
        a, b = int(offsets[m]), int(offsets[m + 1])
        if b <= a:
            continue
        R, t = OG.relative_pose(vms[i], vms[j])
        E = OG.skew(t) @ R
        x = np.stack([(matches[a:b, 0] - intr[i, 2]) / intr[i, 0], (matches[a:b, 1] - intr[i, 3]) / intr[i, 1],
                      np.ones(b - a)], 1)
        y = np.stack([(matches[a:b, 2] - intr[j, 2]) / intr[j, 0], (matches[a:b, 3] - intr[j, 3]) / intr[j, 1],
                      np.ones(b - a)], 1)
        mm = x @ E.T
        n = np.hypot(mm[:, 0] / intr[j, 0], mm[:, 1] / intr[j, 1])
        S = np.abs(y) @ (np.abs(E) + np.linalg.norm(t)) * np.abs(x)
        out[a:b] = S.sum(1) / np.maximum(n, 1e-30)
    return out


def _run_gpu(ii, iv, pairs, M, weights=None, grads=True):
    intr, vm, pr, offs, mt = _cuda(ii, iv, pairs, M.offsets, M.matches)
    w = _cuda(weights.astype(np.float32))[0] if weights is not None else None
    n = len(ii)
    cam_offsets, cam_pairs, status = ga.incidence(pr, n)
    prob = _lib.ga_problem(intr, vm, pr, offs, mt, w)
    dist = torch.empty(len(M.matches), device="cuda")
    sums = torch.empty(max(1, len(pairs)), _lib.GS_GA_PAIR_FLOATS, device="cuda")
    loss = torch.empty(1, device="cuda")
    d_intr = torch.full((n, 4), float("nan"), device="cuda") if grads else None
    d_vm = torch.full((n, 12), float("nan"), device="cuda") if grads else None
    _lib.gs_ga_epipolar(prob, sums, loss, dist=dist, cam_offsets=cam_offsets, cam_pairs=cam_pairs,
                        d_intrinsics=d_intr, d_viewmats=d_vm, status=status)
    torch.cuda.synchronize()
    assert status.cpu().numpy()[0] == 0
    return (dist.cpu().numpy(), float(loss.item()), d_intr.cpu().numpy() if grads else None,
            d_vm.cpu().numpy() if grads else None, cam_offsets.cpu().numpy(), cam_pairs.cpu().numpy())


def _check_distances(e_gpu, e_or, kappa):
    tol = 32 * U32 * kappa + 1e-5 * e_or
    bad = np.abs(e_gpu - e_or) > tol
    assert not bad.any(), (int(bad.sum()), np.abs(e_gpu - e_or)[bad][:5], tol[bad][:5])
    return tol


def test_pair_selection_bit_exact():
    for n, seed in ((300, 0), (57, 3)):
        _, _, iv, _ = synth.ga_cameras(seed, n)
        got = ga.select_pairs(torch.as_tensor(iv).cuda()).cpu().numpy()
        ref = OG.select_pairs(iv, 30.0)
        assert got.shape == ref.shape and (got == ref).all()
    # orbit 12 degrees apart, and a wider threshold
    mats = np.asarray(synth.orbit_viewmats(30), np.float32).reshape(30, 12)
    for deg in (30.0, 50.0):
        got = ga.select_pairs(torch.as_tensor(mats).cuda(), deg).cpu().numpy()
        assert (got == OG.select_pairs(mats, deg)).all()
    # single camera: no pairs; capacity overflow reported, nothing written
    assert ga.select_pairs(torch.as_tensor(mats[:1]).cuda()).shape == (0, 2)
    with pytest.raises(_lib.GsError):
        ga.select_pairs(torch.as_tensor(mats).cuda(), 30.0, capacity=10)


def test_incidence_lists_sorted_and_complete():
    _, _, iv, _ = synth.ga_cameras(0, 120)
    pairs = OG.select_pairs(iv, 30.0)
    offs, lists, status = ga.incidence(torch.as_tensor(pairs).cuda(), 120)
    torch.cuda.synchronize()
    offs, lists = offs.cpu().numpy(), lists.cpu().numpy()
    assert status.cpu().numpy()[0] == 0
    for c in range(120):
        ref = sorted([2 * m for m in np.nonzero(pairs[:, 0] == c)[0]] +
                     [2 * m + 1 for m in np.nonzero(pairs[:, 1] == c)[0]])
        assert list(lists[offs[c]:offs[c + 1]]) == ref


def test_distances_loss_and_gradients_match_the_oracle():
    tv, ti, iv, ii, pairs, M = _problem()
    w = np.random.default_rng(3).uniform(0.1, 2.0, len(M.matches)).astype(np.float32)
    e_or = OG.distances(ii, iv, pairs, M.offsets, M.matches)
    kappa = _kappa(ii.astype(np.float64), iv.astype(np.float64), pairs, M.offsets, M.matches.astype(np.float64))
    tol = 32 * U32 * kappa + 1e-5 * e_or
    # where the sign of x'^T F x is within float32 rounding of 0 the two sides
    # may take different branches of |.|: those matches get weight 0
    w[e_or <= 4 * tol] = 0.0
    e_gpu, L, d_intr, d_vm, _, _ = _run_gpu(ii, iv, pairs, M, w)
    _check_distances(e_gpu, e_or, kappa)
    assert (w == 0).mean() < 0.01
    L_or, di_or, dv_or = OG.loss_and_grads(ii, iv, pairs, M.offsets, M.matches, w)
    assert abs(L - L_or) <= 1e-5 * L_or
    check_grad(d_intr, di_or, "dL/d(fx, fy, cx, cy)")
    check_grad(d_vm, dv_or, "dL/d(R, t)")


def test_weights_counts_and_median_bit_exact():
    tv, ti, iv, ii, pairs, M = _problem(n_views=30, per_pair=500, seed=2, ragged=False)
    e32 = OG.distances(ii, iv, pairs, M.offsets, M.matches).astype(np.float32)
    for n_bins, alpha, sub in ((100, 0.5, len(e32)), (37, 1.0, len(e32) - 1), (4096, 0.5, 1001)):
        e = e32[:sub]
        w, counts, stats = ga.pdf_weights(torch.as_tensor(e).cuda(), n_bins, alpha)
        torch.cuda.synchronize()
        w_or, c_or = OG.pdf_weights(e, n_bins, alpha)
        assert (counts.cpu().numpy().astype(np.int64) == c_or).all()
        assert np.allclose(w.cpu().numpy(), w_or, rtol=2e-6, atol=0)
        lo, hi, _ = OG.median_order_stats(e)
        st = stats.cpu().numpy()
        assert st[0] == e.max() and st[1] == np.float32(lo) and st[2] == np.float32(hi)


def test_weights_edge_cases():
    # all distances zero: one bin, weight 1; a single distance; ties
    for e in (np.zeros(9, np.float32), np.array([3.5], np.float32), np.array([1, 1, 1, 2, 2], np.float32)):
        w, counts, stats = ga.pdf_weights(torch.as_tensor(e).cuda(), 10, 0.5)
        torch.cuda.synchronize()
        w_or, c_or = OG.pdf_weights(e, 10, 0.5)
        assert (counts.cpu().numpy() == c_or).all()
        assert np.allclose(w.cpu().numpy(), w_or, rtol=2e-6)
        lo, hi, _ = OG.median_order_stats(e)
        assert stats.cpu().numpy()[1] == lo and stats.cpu().numpy()[2] == hi


def test_epipolar_edge_cases():
    # no pairs: loss 0, gradients 0
    _, ti, _, _ = synth.ga_cameras(0, 4)
    vm = np.asarray(synth.orbit_viewmats(4), np.float32).reshape(4, 12)
    empty = synth.Matches(np.zeros(1, np.int64), np.zeros((0, 4), np.float32), np.zeros(0, bool))
    _, L, d_intr, d_vm, _, _ = _run_gpu(ti, vm, np.zeros((0, 2), np.int32), empty)
    assert L == 0 and not d_intr.any() and not d_vm.any()
    # coincident camera centres at the origin (t_i = t_j = 0, so t_ij = 0 and
    # F = 0 exactly in float32 too): every distance 0, no gradient
    vm2 = np.zeros((2, 12), np.float32)
    vm2[0, :9] = synth.look_at((0.0, 0.0, -5.0))[:9]
    vm2[1, :9] = synth.look_at((3.0, 0.0, -4.0))[:9]
    pairs = np.array([[0, 1]], np.int32)
    M = synth.Matches(np.array([0, 5], np.int64), np.random.default_rng(0).uniform(0, 900, (5, 4)).astype(np.float32),
                      np.ones(5, bool))
    e, L, d_intr, d_vm, _, _ = _run_gpu(ti[:2], vm2, pairs, M)
    assert not e.any() and L == 0 and not d_intr.any() and not d_vm.any()
    assert not OG.distances(ti[:2], vm2, pairs, M.offsets, M.matches).any()
    L_or, di, dv = OG.loss_and_grads(ti[:2], vm2, pairs, M.offsets, M.matches)
    assert L_or == 0 and not di.any() and not dv.any()


def test_full_size_parity():
    """The bench's configuration: 300 cameras, pairs within 30 degrees,
    4,096 matches per pair with 15 % outliers, Eq. 3 weights; every
    distance, the loss and every camera gradient."""
    tv, ti, iv, ii = synth.ga_cameras(0)
    pairs_gpu = ga.select_pairs(torch.as_tensor(iv).cuda())
    pairs = OG.select_pairs(iv, 30.0)
    assert (pairs_gpu.cpu().numpy() == pairs).all()
    M = synth.ga_matches(1, synth.ga_points(0), ti, tv, pairs, 1600, 1066)
    assert len(M.matches) > 20_000_000
    e_or = OG.distances(ii, iv, pairs, M.offsets, M.matches)
    e32 = e_or.astype(np.float32)
    w_or, _ = OG.pdf_weights(e32, 100, 0.5)
    w, counts, stats = ga.pdf_weights(torch.as_tensor(e32).cuda(), 100, 0.5)
    torch.cuda.synchronize()
    assert np.allclose(w.cpu().numpy(), w_or, rtol=2e-6)
    w = w.cpu().numpy()
    kappa = _kappa(ii.astype(np.float64), iv.astype(np.float64), pairs, M.offsets, M.matches.astype(np.float64))
    tol = 32 * U32 * kappa + 1e-5 * e_or
    w[e_or <= 4 * tol] = 0.0
    e_gpu, L, d_intr, d_vm, _, _ = _run_gpu(ii, iv, pairs, M, w)
    _check_distances(e_gpu, e_or, kappa)
    L_or, di_or, dv_or = OG.loss_and_grads(ii, iv, pairs, M.offsets, M.matches, w)
    assert abs(L - L_or) <= 1e-5 * L_or
    check_grad(d_intr, di_or, "full size dL/d(fx, fy, cx, cy)")
    check_grad(d_vm, dv_or, "full size dL/d(R, t)")


def _rel_rot_err(vm_a, vm_b, pairs):
    """Mean angle (degrees) between the relative rotations of the pairs."""
    out = []
    for i, j in pairs:
        Ra, _ = OG.relative_pose(vm_a[i], vm_a[j])
        Rb, _ = OG.relative_pose(vm_b[i], vm_b[j])
        c = (np.trace(Ra @ Rb.T) - 1) / 2
        out.append(np.degrees(np.arccos(np.clip(c, -1, 1))))
    return float(np.mean(out))


def test_alignment_reduces_pose_error():
    tv, ti, iv, ii = synth.ga_cameras(5, 60)
    pairs = OG.select_pairs(iv, 30.0)
    M = synth.ga_matches(5, synth.ga_points(5, 8000), ti, tv, pairs, 1600, 1066, 1500)
    intr, vm, pr, offs, mt = _cuda(ii, iv, pairs, M.offsets, M.matches)
    G = ga.GlobalAlignment(intr, vm, pr, offs, mt)
    assert G.lr in ga.LRS
    e0 = _rel_rot_err(tv.astype(np.float64), iv.astype(np.float64), pairs)
    intr1, vm1 = G.run(300)
    torch.cuda.synchronize()
    G.check()
    vm1 = vm1.detach().cpu().numpy().astype(np.float64)
    e1 = _rel_rot_err(tv.astype(np.float64), vm1, pairs)
    d1 = OG.distances(intr1.detach().cpu().numpy(), vm1, pairs, M.offsets, M.matches)
    d0 = OG.distances(ii, iv, pairs, M.offsets, M.matches)
    assert np.median(d1[M.inlier]) < 0.5 * np.median(d0[M.inlier]), (np.median(d0[M.inlier]), np.median(d1[M.inlier]))
    assert e1 < 0.5 * e0, (e0, e1)


def test_fused_step_matches_the_oracle_chain():
    """gs_ga_step: cameras from residuals, residual gradients through the
    Gram-Schmidt chain and the Adam update, each against the FP64 oracle, over
    two calls (the device step counter drives the bias correction)."""
    from oracle.optim import adam_sgld_step
    tv, ti, iv, ii, pairs, M = _problem(n_views=30, per_pair=600, seed=4)
    n = len(iv)
    rng = np.random.default_rng(9)
    res = np.tile(np.array([1, 0, 0, 0, 1, 0, 0, 0, 0, 0], np.float32), (n, 1))
    res += (0.02 * rng.standard_normal((n, 10))).astype(np.float32)
    w = rng.uniform(0.1, 2.0, len(M.matches)).astype(np.float32)
    intr0, vm0, pr, offs, mt, wt, r = _cuda(ii, iv, pairs, M.offsets, M.matches, w, res)
    m = torch.zeros_like(r)
    v = torch.zeros_like(r)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    intr = torch.empty_like(intr0)
    vm = torch.empty_like(vm0)
    cam_offsets, cam_pairs, status = ga.incidence(pr, n)
    lr = 1e-3
    state = _lib.ga_state(intr0, vm0, r, m, v, step, intr, vm, lr)
    sums = torch.empty(len(pairs), _lib.GS_GA_PAIR_FLOATS, device="cuda")
    loss = torch.empty(1, device="cuda")
    d_res = torch.empty_like(r)
    groups = [dict(param=res.astype(np.float64), grad=None, m=np.zeros((n, 10)), v=np.zeros((n, 10)), lr=lr)]
    for call in (1, 2):
        res_before = r.cpu().numpy().astype(np.float64)
        # mask matches whose |x'^T F x| is within float32 rounding of 0 at the
        # cameras of this call (computed from the oracle's cameras)
        i_or, v_or = OG.apply_residuals(ii, iv, res_before)
        e_or = OG.distances(i_or, v_or, pairs, M.offsets, M.matches)
        kappa = _kappa(i_or, v_or, pairs, M.offsets, M.matches.astype(np.float64))
        wm = w.copy()
        wm[e_or <= 4 * (32 * U32 * kappa + 1e-5 * e_or)] = 0.0
        wt.copy_(torch.as_tensor(wm))
        prob = _lib.ga_problem(intr, vm, pr, offs, mt, wt)
        _lib.gs_ga_step(state, prob, sums, cam_offsets, cam_pairs, loss, d_res, status)
        torch.cuda.synchronize()
        assert status.cpu().numpy()[0] == 0 and int(step.item()) == call
        # cameras
        assert np.allclose(vm.cpu().numpy(), v_or, rtol=0, atol=2e-6 * np.abs(v_or).max())
        assert np.allclose(intr.cpu().numpy(), i_or, rtol=1e-6)
        # loss and residual gradients at the GPU's cameras
        gi, gv = intr.cpu().numpy().astype(np.float64), vm.cpu().numpy().astype(np.float64)
        L_or, di, dv = OG.loss_and_grads(gi, gv, pairs, M.offsets, M.matches, wm)
        assert abs(float(loss.item()) - L_or) <= 1e-5 * L_or
        g_or = OG.residual_vjp(ii, iv, res_before, di, dv)
        g_gpu = d_res.cpu().numpy()
        check_grad(g_gpu, g_or, f"call {call}: dL/d(residuals)")
        # Adam update from the GPU's gradient, in FP64
        groups[0]["param"] = res_before.copy()
        groups[0]["grad"] = g_gpu.astype(np.float64)
        adam_sgld_step(groups, call, 0.9, 0.999, 1e-15)
        assert np.allclose(r.cpu().numpy(), groups[0]["param"], rtol=0, atol=1e-6)
        assert np.allclose(m.cpu().numpy(), groups[0]["m"], rtol=1e-5, atol=1e-7 * np.abs(groups[0]["m"]).max())


def test_unfused_iteration_converges_like_the_fused_one():
    tv, ti, iv, ii = synth.ga_cameras(6, 40)
    pairs = OG.select_pairs(iv, 30.0)
    M = synth.ga_matches(6, synth.ga_points(6, 6000), ti, tv, pairs, 1600, 1066, 1000)
    intr, vm, pr, offs, mt = _cuda(ii, iv, pairs, M.offsets, M.matches)
    e0 = _rel_rot_err(tv.astype(np.float64), iv.astype(np.float64), pairs)
    out = []
    for fused in (True, False):
        G = ga.GlobalAlignment(intr, vm, pr, offs, mt, fused=fused)
        _, vm1 = G.run(150)
        torch.cuda.synchronize()
        G.check()
        out.append(_rel_rot_err(tv.astype(np.float64), vm1.detach().cpu().numpy().astype(np.float64), pairs))
    assert out[0] < 0.3 * e0 and out[1] < 0.3 * e0, (e0, out)
