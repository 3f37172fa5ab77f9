#!/usr/bin/env python
"""Throughput of the differentiable 3DGS rasterizer with pose gradients.

One step = project + bin/sort + render forward + L1 loss + raster backward +
projection backward + pose-gradient reduction over one batch of views, i.e.
forward and backward to every Gaussian parameter and every view's pose.

Default workload: 1,000,000 clustered SH-degree-3 Gaussians, one 1237x822
view (fx=fy=1000), synthetic and seeded; the step is captured once into a
CUDA graph and replayed. Metric: pixels per second (Mpix/s) of fwd+bwd incl.
pose gradients; ``value`` is the whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the path has no exchange step on one GPU per process): weak
scaling, max-over-ranks time. ``--impl reference`` times the FP64 CPU oracle
on the host cores (rank 0 only) on bounded pixel samples of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpix/s incl. pose grads at 1M Gaussians"
UNIT = "Mpix/s"

# FP32 operations per pixel-Gaussian pair. The method's count: about 12
# flops + 1 ex2 per evaluated pair in the forward and 40 flops + 1 ex2 in the
# backward. The kernels' own arithmetic (gs_render.cu): every pair that
# passes the pixel gate evaluates the exponent (dx, dy, 3 mul + 2 fma, o*G,
# clamp/threshold: 10 ops + 1 ex2); a composited pair adds 9 in the forward
# (1-alpha, T update, weight, 3 fma) and 50 in the backward (colour/alpha/
# conic/mean gradients and the recomputed accumulation).
FWD_FLOPS_EVAL, BWD_FLOPS_EVAL = 12, 40
FWD_OPS_EVAL, FWD_OPS_COMP = 10, 9
BWD_OPS_EVAL, BWD_OPS_COMP = 10, 50
FP32_LANES_PER_SM = 128
# tile shapes the autotuner tries on the large secondary workloads (uneven
# scenes, dense step), where each candidate step is expensive to build: the
# shapes that won on any workload measured so far (every batch is tried)
SECONDARY_TILES = ((16, 16), (32, 16), (32, 32))


# DRAM traffic per launch of the raster backward (dram__bytes_read.sum +
# dram__bytes_write.sum, mean of three launches of one ncu capture of this
# workload). It holds only for the kernel source it was measured on (hash of
# its two source files) and for the default workload, tile and backward
# batch; otherwise the bench reports null.
RASTER_BWD_TRAFFIC = {"bytes": 56664234, "sources_sha256_16": "90592951efb75907", "n": 1_000_000,
                      "tile": (32, 32), "bwd_batch": 1}


def raster_bwd_sources_hash():
    import hashlib
    h = hashlib.sha256()
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2509_25191_gb300", "csrc")
    for f in ("gs_render.cu", "gs_common.cuh"):
        with open(os.path.join(here, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--tile", default="auto", help="tile shape WxH, or auto (the project's autotuner picks the "
                                                   "tile and the shared-memory batch)")
    ap.add_argument("--batch", default="2,1", help="with a fixed --tile: Gaussians per thread per shared-memory "
                                                   "batch, forward,backward")
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-ga", action="store_true", help="skip the global-alignment workload")
    ap.add_argument("--only", choices=["ga", "oracle_views"], default=None,
                    help="run only the named secondary workload and print its figures (for profiling); "
                         "oracle_views times the FP64 oracle on one view of each configuration")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the uneven multi-scene batch and the dense-view joint pose step")
    ap.add_argument("--ref-fraction", type=float, default=1.0,
                    help="pixel fraction of each reference-arm step (1 = the whole workload, the same "
                         "configuration as the native arm)")
    return ap.parse_args()


def workload(n):
    from paper_2509_25191_gb300 import synth
    sc, vw = synth.single_view_1m(0, n)
    return sc, vw


def stage_bytes(n, sh_degree, slots, instances, pixels, n_tiles):
    """Bytes each stage of the method must move per step (the raw record
    R_in = 236 B for SH3): projection reads the records once for all views
    and writes a 48-B record and a 4-B tile count per slot; binning writes
    the instance list (12 B) and reads it sorted once, plus the tile ranges;
    the forward gathers each instance's 36-B payload and 4-B id and writes the
    image (12 B per pixel); the backward gathers them again (40 B), reads the
    image and its gradient (24 B per pixel) and writes and reads the 2D
    gradients (80 B per slot); the projection backward re-reads the records
    and writes their gradients."""
    r_in = 4 * (3 + 3 + 4 + 1 + 3 * (sh_degree + 1) ** 2)
    return {"gs_project": n * r_in + 52 * slots,
            "gs_bin_sort": 24 * instances + 8 * n_tiles,
            "gs_render_fwd": 40 * instances + 12 * pixels,
            "gs_rasterize_bwd": 40 * instances + 24 * pixels + 40 * slots,
            "gs_project_bwd": 2 * n * r_in + 40 * slots}


def algorithmic_bytes(n, sh_degree, slots, instances, pixels, n_tiles):
    """Bytes the method must move per step: raw records read twice and
    gradients written once (3 N R_in), projected records written and read
    (64 + 48 B per slot for records and 2D gradients, both ways 132 B),
    tile instances (key + id written, read sorted, gathered in forward and
    backward: 108 B), images (colour, target, upstream, image re-read: 36 B
    per pixel), tile ranges."""
    r_in = 4 * (3 + 3 + 4 + 1 + 3 * (sh_degree + 1) ** 2)
    return 3 * n * r_in + 132 * slots + 108 * instances + 36 * pixels + 8 * n_tiles


def measure_alu_peaks(dev, iters=16384, launches=60):
    """Measured arithmetic throughput of one GB300 (CUDA events, after warm-up):
    scalar FP32 FMA, packed f32x2 FMA and ex2.approx, from the library's probe
    kernels, with the SM clock sampled meanwhile; FMA rates in FLOP/s (2 per
    FMA), ex2 in operations/s, and each per SM and clock cycle."""
    import torch

    from paper_2509_25191_gb300 import _lib
    out = None
    res = {}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    with ClockSampler(dev.index or 0) as clk:
        for kind, name in ((0, "fp32_fma"), (1, "fp32_fma_f32x2"), (2, "ex2")):
            for _ in range(3):
                out, ops = _lib.gs_peak_probe(kind, iters, out)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(launches):
                _lib.gs_peak_probe(kind, iters, out)
            b.record()
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) * 1e-3 / launches
            res[name] = ops / sec * (1 if kind == 2 else 2)
    clocks = clk.summary()
    mhz = clocks.get("sm_mhz") or 2070.0
    out = {k: round(v / 1e12, 3) for k, v in res.items()}
    out["unit"] = "TFLOP/s (ex2: T ops/s)"
    out["per_sm_per_clock"] = {k: round(v / (sms * mhz * 1e6), 2) for k, v in res.items()}
    out["fp32_peak_tflops"] = round(max(res["fp32_fma"], res["fp32_fma_f32x2"]) / 1e12, 3)
    out["clocks"] = clocks
    return out


class ClockSampler:
    """nvidia-smi samples (every 100 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, v in enumerate(fl) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value, device=None):
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix_s(pixels_per_rank, world, ms_per_step):
    """Whole-job throughput of N replicas, each doing pixels_per_rank per step."""
    return world * pixels_per_rank / (ms_per_step * 1e-3) / 1e6


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------

def run_native(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2509_25191_gb300 import _lib, build
    from paper_2509_25191_gb300.step import GraphStep

    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    sc, vw = workload(args.n)
    g = _lib.Gaussians.from_scene(sc, dev)
    views = _lib.Views.from_synth(vw, dev)
    P = views.pixels
    rng = np.random.default_rng(1234)
    target = torch.as_tensor(rng.uniform(0, 1, views.num_image_floats()).astype(np.float32), device=dev)
    tuning = None
    if args.tile == "auto":
        from paper_2509_25191_gb300.tune import autotune, key_str
        choice, ms = autotune(g, views, target)
        tile, batch = choice.tile, choice.batch
        tuning = {"chosen": {"tile": list(tile), "batch": list(batch)},
                  "ms_per_step": {key_str(c): round(v, 4) for c, v in sorted(ms.items(), key=lambda kv: kv[1])},
                  "key": "tile WxH / Gaussians per thread per shared-memory batch (forward.backward)"}
    else:
        tile = tuple(int(x) for x in args.tile.split("x"))
        batch = tuple(int(x) for x in args.batch.split(","))

    # two input slots (target, view matrices): the end-to-end loop below
    # uploads step k+1's inputs into one while step k runs on the other
    step = GraphStep(g, views, target, tile=tile, batch=batch, slots=2, slot_gaussians=not args.no_e2e)
    rast, cfg, bins = step.rast, step.cfg, step.bins
    image, dvm, loss = step.image, step.dviewmat, step.loss
    kernels_per_step = step.kernels_per_step()
    torch.cuda.synchronize()
    rast.check_status()

    # per-stage durations (CUDA events on the launching stream, eager calls)
    names = list(step.stages)
    acc = np.zeros(len(names))
    reps = 10
    for _ in range(reps):
        ev = []
        step.run(ev)
        torch.cuda.synchronize()
        acc += [ev[i].elapsed_time(ev[i + 1]) for i in range(len(names))]
    stage_ms = acc / reps
    # pixel-Gaussian pair counts of the raster backward: one extra eager step
    # with counting switched on (the timed step does not count)
    step.cfg.count_pairs = 1
    step.run()
    torch.cuda.synchronize()
    pairs = _lib.pair_counts(bins)
    step.cfg.count_pairs = 0
    n_inst = int(bins.counters[0].item())

    graph = step.graph
    for _ in range(max(3, args.warmup)):
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream()
        t0.record(cur)
        for _ in range(args.steps):
            graph.replay()
        t1.record(cur)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1) / args.steps, dev)
    clocks = clk.summary()
    rast.check_status()
    value = whole_job_mpix_s(P, world, ms)

    # end to end through the public API, each step fed from pinned host memory.
    # e2e: a training step with the Gaussians resident on the device (the model
    # state): the step's target image and camera pose are copied in, the loss
    # and the pose gradient read back. e2e_params_in: the same, plus all
    # Gaussian parameters copied in and the rendered image read back each step.
    e2e = None
    e2e_params = None
    if not args.no_e2e:
        k_e2e = max(3, min(args.steps, 50))
        tgt_dev = step.target
        host_step = [tgt_dev.cpu().pin_memory(), views.viewmats.cpu().pin_memory()]
        host_par = [t.cpu().pin_memory() for t in (g.means, g.log_scales, g.quats, g.opacity_logits, g.sh)]
        out_img = torch.empty(image.shape, dtype=torch.float32).pin_memory()
        out_pose = torch.empty(dvm.shape, dtype=torch.float32).pin_memory()
        out_loss = torch.empty(loss.shape, dtype=torch.float32).pin_memory()

        # step k+1's inputs (the target image and the view matrices) are
        # uploaded on a copy stream into the step's other input slot while
        # step k computes; each step's graph reads its own slot
        copy_stream = torch.cuda.Stream(device=dev)
        ready = [torch.cuda.Event() for _ in range(2)]
        consumed = [torch.cuda.Event() for _ in range(2)]
        # step k's loss and pose gradient (kept per slot by the step) are read
        # back on another stream while step k+1 runs; the next replay of the
        # slot waits until they have been read
        d2h_stream = torch.cuda.Stream(device=dev)
        done = [torch.cuda.Event() for _ in range(2)]
        read = [torch.cuda.Event() for _ in range(2)]
        main = torch.cuda.current_stream(dev)

        def run_e2e(with_params):
            hosts = host_par if with_params else []
            outs = [(out_loss, loss), (out_pose, dvm)] + ([(out_img, image)] if with_params else [])
            state = {"k": 0}

            def upload(k):
                sl = k % 2
                gs = step.gauss_slots[sl]
                with torch.cuda.stream(copy_stream):
                    copy_stream.wait_event(consumed[sl])      # the step that last read this slot is done
                    step.viewmat_slots[sl].copy_(host_step[1], non_blocking=True)
                    step.target_slots[sl].copy_(host_step[0], non_blocking=True)
                    for h, d in zip(hosts, (gs.means, gs.log_scales, gs.quats, gs.opacity_logits, gs.sh)):
                        d.copy_(h, non_blocking=True)
                    ready[sl].record(copy_stream)

            upload(0)

            def e2e_step():
                k = state["k"]
                sl = k % 2
                main.wait_event(ready[sl])
                main.wait_event(read[sl])
                upload(k + 1)
                step.replay(sl)
                consumed[sl].record(main)
                if with_params:
                    out_img.copy_(image, non_blocking=True)   # (one image buffer for both slots)
                done[sl].record(main)
                with torch.cuda.stream(d2h_stream):
                    d2h_stream.wait_event(done[sl])
                    out_loss.copy_(step.loss_slots[sl], non_blocking=True)
                    out_pose.copy_(step.dviewmat_slots[sl], non_blocking=True)
                    read[sl].record(d2h_stream)
                state["k"] = k + 1

            for _ in range(3):
                e2e_step()
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(k_e2e):
                e2e_step()
            main.wait_stream(d2h_stream)   # the last step's results are read inside the timed region
            b.record()
            torch.cuda.synchronize()
            ems = max_over_ranks(a.elapsed_time(b) / k_e2e, dev)
            return {"value": round(whole_job_mpix_s(P, world, ems), 3), "unit": UNIT,
                    "h2d_bytes_per_step": int(sum(h.numel() * 4 for h in host_step + hosts)),
                    "d2h_bytes_per_step": int(sum(o.numel() * 4 for o, _ in outs)),
                    "ms_per_step": round(ems, 4), "steps": k_e2e}

        e2e = run_e2e(False)
        e2e["inputs"] = ("target image and camera pose in, loss and pose gradient out; Gaussians resident; "
                         "the next step's target and pose upload on a copy stream into the step's other "
                         "input slot during the current step, and the step's loss and pose gradient (kept "
                         "per slot) are read back on a third stream during the next step")
        e2e_params = run_e2e(True)
        e2e_params["inputs"] = ("also all Gaussian parameters in (uploaded with the step's other inputs into "
                                "its other slot) and the rendered image out, every step")

    # roofline of the dominant kernel
    rt = RASTER_BWD_TRAFFIC
    # (the forward's batch does not change the backward kernel)
    raster_traffic = rt["bytes"] if (args.n == rt["n"] and tuple(tile) == rt["tile"] and batch[1] == rt["bwd_batch"]
                                     and raster_bwd_sources_hash() == rt["sources_sha256_16"]) else None
    peaks, peak_src = measured_peaks()
    alu = measure_alu_peaks(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    top = int(np.argmax(stage_ms))
    t_top = stage_ms[top] * 1e-3
    if names[top] in ("gs_render_fwd", "gs_rasterize_bwd", "gs_rasterize_bwd_l1"):
        fwd = names[top] == "gs_render_fwd"
        ev_, co_ = (pairs[0], pairs[1]) if fwd else (pairs[2], pairs[3])
        flops = (FWD_FLOPS_EVAL if fwd else BWD_FLOPS_EVAL) * ev_
        kops = (FWD_OPS_EVAL * ev_ + FWD_OPS_COMP * co_) if fwd else (BWD_OPS_EVAL * ev_ + BWD_OPS_COMP * co_)
        peak = alu["fp32_peak_tflops"]
        achieved = flops / t_top / 1e12
        nominal = sms * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"kernel": names[top], "bound": "alu", "achieved": round(achieved, 3), "peak": peak,
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": raster_traffic,
                "peak_source": "measured: FP32 FMA probe kernels of this library on this GPU (best of scalar and "
                               "packed f32x2), CUDA events, clocks sampled (alu_peaks)",
                "ops_basis": f"{FWD_FLOPS_EVAL if fwd else BWD_FLOPS_EVAL} FP32 flops per evaluated pixel-Gaussian "
                             "pair (the method's count)",
                "units": {"pairs_evaluated": ev_, "pairs_composited": co_, "fp32_flops": int(flops)},
                "kernel_ops": {"ops": int(kops), "basis": "the kernel's own arithmetic: "
                               f"{BWD_OPS_EVAL if not fwd else FWD_OPS_EVAL} per evaluated + "
                               f"{BWD_OPS_COMP if not fwd else FWD_OPS_COMP} per composited pair",
                               "achieved": round(kops / t_top / 1e12, 3),
                               "frac": round(kops / t_top / 1e12 / peak, 4)},
                "nominal_peak": {"value": round(nominal, 2),
                                 "basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                          f"{peaks.get('sm_max_mhz', 2070.0)} MHz"}}
    else:
        hbm = peaks["hbm_gbs"]
        roof = {"kernel": names[top], "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
                "traffic": None}
    # the same step with the L1 + D-SSIM loss of Section 3.1 (fused kernel), and that kernel alone
    dstep = GraphStep(g, views, target, tile=tile, batch=batch, loss="l1_dssim")
    dssim = {"ms_per_step": round(_time_replays(dstep, 50), 4)}
    dssim["mpix_s"] = round(P / dssim["ms_per_step"] / 1e3, 2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(20):
        _lib.gs_l1_dssim_loss(views, dstep.image, dstep.target, dstep.loss, dstep.dimg, 0.2)
    ev1.record()
    torch.cuda.synchronize()
    dssim["loss_kernel_ms"] = round(ev0.elapsed_time(ev1) / 20, 4)
    dssim["loss"] = [round(float(v), 6) for v in dstep.loss.cpu()]
    del dstep
    # the small configuration (2,000 SH0 Gaussians, one 128x128 view), captured the same way
    from paper_2509_25191_gb300 import synth as _synth
    ssc, svw = _synth.single_view_small()
    sg = _lib.Gaussians.from_scene(ssc, dev)
    sv = _lib.Views.from_synth(svw, dev)
    sstep = GraphStep(sg, sv, torch.rand(sv.num_image_floats(), device=dev, generator=torch.Generator(dev).manual_seed(3)),
                      tile=(16, 16))
    small = {"workload": "2,000 SH0 Gaussians uniform in a box, one 128x128 view, fwd+L1+bwd+pose, 16x16 tiles",
             "ms_per_step": round(_time_replays(sstep, 200), 4)}
    small["mpix_s"] = round(sv.pixels / small["ms_per_step"] / 1e3, 2)
    del sstep
    # test-time pose tuning (Gaussians frozen): the same step with the backward to the pose only
    pstep = GraphStep(g, views, target, tile=tile, batch=batch, want_gaussian_grads=False)
    pose_only = {"ms_per_step": round(_time_replays(pstep, 50), 4)}
    pose_only["mpix_s"] = round(P / pose_only["ms_per_step"] / 1e3, 2)
    del pstep
    batched = None if args.no_batched else batched_vs_plain(dev, (tile, batch) if args.tile != "auto" else "auto")
    extra = {} if args.no_extra else {"uneven_scenes": run_uneven(dev), "dense_pose_step": run_dense(dev)}
    if not args.no_ga:
        extra["ga_epipolar"] = run_ga(dev)
    extra = extra or None
    step_bytes = algorithmic_bytes(g.n, g.sh_degree, views.num_slots(), n_inst, P, views.num_tiles(cfg))
    hbm_frac_step = step_bytes / (ms * 1e-3) / (peaks["hbm_gbs"] * 1e9)
    sb = stage_bytes(g.n, g.sh_degree, views.num_slots(), n_inst, P, views.num_tiles(cfg))
    # (the raster backward with the L1 loss folded in reads the target where
    # the plain one reads dL/dimage: the same bytes)
    sb["gs_rasterize_bwd_l1"] = sb["gs_rasterize_bwd"]
    stage_frac = {n: {"algorithmic_bytes": int(sb[n]), "ms": round(float(t), 4),
                      "frac_of_hbm": round(sb[n] / (float(t) * 1e-3) / (peaks["hbm_gbs"] * 1e9), 4)}
                  for n, t in zip(names, stage_ms) if n in sb}

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"single view 1237x822, {g.n} clustered SH3 Gaussians (seed 0), fwd+L1+bwd+pose",
                   "gaussians": g.n, "views": views.n, "pixels_per_step": P, "tile": list(tile), "batch": list(batch),
                   "instances": n_inst, "l2": "inputs larger than L2 (236 MB raw records + 64 MB projected)",
                   "graph": "one CUDA graph per step", "parallelism": f"replicas x{world}"},
        "roofline": roof,
        "step_hbm_roofline": {"algorithmic_bytes": int(step_bytes), "frac": round(hbm_frac_step, 4),
                              "peak_gbs": peaks["hbm_gbs"], "peak_source": peak_src},
        "stages_ms": {n: round(float(t), 4) for n, t in zip(names, stage_ms)},
        "stage_hbm_roofline": stage_frac,
        "alu_peaks": alu,
        "autotune": tuning,
        "clocks": clocks,
        "pose_only_step": pose_only,
        "small_case": small,
        "l1_dssim_step": dssim,
        "batched_vs_plain": batched,
        "other_workloads": extra,
        "e2e": e2e,
        "e2e_params_in": e2e_params,
        "gpu_launches": kernels_per_step * args.steps,
    }
    return out, sc, vw


def batched_vs_plain(dev, tile, steps=20, plain_steps=5):
    """16 views 979x546 of one 500K-Gaussian clustered SH3 scene on a circular
    orbit: the whole batch in one captured step versus the same work as 16
    uncaptured single-view calls (each with its instance-count readback)."""
    import torch

    from paper_2509_25191_gb300 import _lib, synth
    from paper_2509_25191_gb300.step import GraphStep, PlainStep
    sc, vw = synth.orbit_views(0, 500_000, 16, 979, 546)
    g = _lib.Gaussians.from_scene(sc, dev)
    views = _lib.Views.from_synth(vw, dev)
    rng = np.random.default_rng(99)
    target = torch.as_tensor(rng.uniform(0, 1, views.num_image_floats()).astype(np.float32), device=dev)
    if tile == "auto":
        from paper_2509_25191_gb300.tune import autotune
        choice, _ = autotune(g, views, target)
        tile, batch = choice.tile, choice.batch
    else:
        tile, batch = tile
    gs = GraphStep(g, views, target, tile=tile, batch=batch)
    ps = PlainStep(g, views, target, tile=tile, batch=batch)
    for _ in range(3):
        gs.replay()
        ps.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        gs.replay()
    b.record()
    torch.cuda.synchronize()
    tb = a.elapsed_time(b) / steps
    gs.rast.check_status()
    a.record()
    for _ in range(plain_steps):
        ps.run()
    b.record()
    torch.cuda.synchronize()
    tp = a.elapsed_time(b) / plain_steps
    px = views.pixels
    # where each arm's time goes: eager per-stage events (the batched step's
    # calls once over all views; the plain arm's calls per view, summed)
    reps = 3
    bn = list(gs.stages)
    bacc = np.zeros(len(bn))
    pacc = np.zeros(len(PlainStep.STAGES))
    for _ in range(reps):
        ev = []
        gs.run(ev)
        torch.cuda.synchronize()
        bacc += [ev[i].elapsed_time(ev[i + 1]) for i in range(len(bn))]
        ev = []
        ps.run(ev)
        torch.cuda.synchronize()
        k = len(PlainStep.STAGES)
        for v in range(len(ev) // (k + 1)):
            e = ev[v * (k + 1):(v + 1) * (k + 1)]
            pacc += [e[i].elapsed_time(e[i + 1]) for i in range(k)]
    bst = {n: round(float(t) / reps, 4) for n, t in zip(bn, bacc)}
    peaks, _ = measured_peaks()
    bbytes = algorithmic_bytes(g.n, g.sh_degree, views.num_slots(), int(gs.bins.counters[0].item()), px,
                               views.num_tiles(gs.cfg))
    pst = {n: round(float(t) / reps, 4) for n, t in zip(PlainStep.STAGES, pacc)}
    return {"workload": "16 views 979x546 on a radius-5 orbit, 500K clustered SH3 Gaussians (seed 0), "
                        "fwd+L1+bwd+pose", "batched_ms": round(tb, 4), "plain_ms": round(tp, 4),
            "tile": list(tile), "batch": list(batch), "batched_mpix_s": round(px / tb / 1e3, 2),
            "plain_mpix_s": round(px / tp / 1e3, 2),
            "ratio": round(tp / tb, 3), "steps": steps, "plain_steps": plain_steps,
            "batched_stages_ms": bst,
            "batched_hbm_roofline": {"algorithmic_bytes": int(bbytes),
                                     "frac": round(bbytes / (tb * 1e-3) / (peaks["hbm_gbs"] * 1e9), 4)},
            "plain_stages_ms": pst,
            "plain_definition": "the same library called view by view, uncaptured, each call with the instance-count "
                                "readback an uncaptured call needs (bin_sort includes it); the same calls as the "
                                "batched step (L1 loss folded into the raster backward, zeroing overlapped with "
                                "the kernel ahead)"}


def _time_replays(step, steps):
    import torch
    for _ in range(3):
        step.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        step.replay()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def run_uneven(dev, steps=10):
    """8 scenes of 0.2M..3M clustered SH3 Gaussians (seeds 1-8), 4 views each
    at mixed resolutions: all 32 views in one captured step."""
    import torch

    from paper_2509_25191_gb300 import _lib, synth
    from paper_2509_25191_gb300.step import GraphStep
    from paper_2509_25191_gb300.tune import autotune
    from paper_2509_25191_gb300.layout import reorder, spatial_order
    sc, vw = synth.uneven_scenes()
    # each scene's Gaussians in spatial (Morton) order, kept in the scene's range
    g = _lib.Gaussians.from_scene(sc, dev)
    ranges = sorted({(int(b), int(c)) for b, c in zip(vw.gauss_begin, vw.gauss_count)})
    g = reorder(g, spatial_order(g.means, ranges))
    views = _lib.Views.from_synth(vw, dev)
    target = torch.rand(views.num_image_floats(), device=dev, generator=torch.Generator(dev).manual_seed(5))
    choice, _ = autotune(g, views, target, tiles=SECONDARY_TILES, reps=3)
    step = GraphStep(g, views, target, tile=choice.tile, batch=choice.batch)
    ms = _time_replays(step, steps)
    step.rast.check_status()
    tile = choice.tile
    peaks, _ = measured_peaks()
    ubytes = algorithmic_bytes(g.n, g.sh_degree, views.num_slots(), int(step.bins.counters[0].item()), views.pixels,
                               views.num_tiles(step.cfg))
    return {"workload": "8 scenes 0.2M-3M SH3 Gaussians (11.7M), 32 views at mixed resolutions, fwd+L1+bwd+pose",
            "gaussians": g.n, "views": views.n, "pixels_per_step": views.pixels, "tile": list(tile),
            "batch": list(choice.batch), "instances": int(step.bins.counters[0].item()), "ms_per_step": round(ms, 3),
            "hbm_roofline": {"algorithmic_bytes": int(ubytes),
                             "frac": round(ubytes / (ms * 1e-3) / (peaks["hbm_gbs"] * 1e9), 4)},
            "mpix_s": round(views.pixels / ms / 1e3, 2)}


def run_dense(dev, steps=10, n=6_000_000, n_views=300, batch=8):
    """Joint pose + 3DGS step: 6M SH3 Gaussians, 300 hemisphere views
    1600x1066 with jittered poses; per step a minibatch of 8 views, 6D +
    translation pose residuals composed in torch, the rasterizer step
    (fwd, L1 against targets rendered from the true poses, full backward)
    replayed from one CUDA graph, and the residual gradients by autograd."""
    import torch

    from paper_2509_25191_gb300 import _lib, pose, synth
    from paper_2509_25191_gb300.autograd import Rasterizer
    from paper_2509_25191_gb300.step import GraphStep
    from paper_2509_25191_gb300.layout import reorder, spatial_order
    sc, true_v, noisy_v = synth.dense_hemisphere(0, n, n_views)
    # the training loop keeps its Gaussians in spatial (Morton) order
    g = _lib.Gaussians.from_scene(sc, dev)
    g = reorder(g, spatial_order(g.means))
    W, H = int(true_v.width[0]), int(true_v.height[0])
    true_vm = torch.as_tensor(true_v.viewmats, device=dev)
    noisy_vm = torch.as_tensor(noisy_v.viewmats, device=dev)
    intr = torch.as_tensor(true_v.intrinsics, device=dev)
    # targets from the unperturbed poses, rendered once by the validated forward
    targets = torch.empty(n_views, 3 * W * H, device=dev)
    rast = Rasterizer()
    for v0 in range(0, n_views, batch):
        ids = list(range(v0, min(n_views, v0 + batch)))
        vv = _lib.Views(true_vm[ids].contiguous(), intr[ids].contiguous(), [W] * len(ids), [H] * len(ids),
                        [0] * len(ids), [n] * len(ids))
        img, _ = rast.forward(g, vv)
        targets[ids] = img.view(len(ids), -1)
    del rast
    dr = pose.identity_6d(n_views, device=dev).requires_grad_(True)
    dt = torch.zeros(n_views, 3, device=dev, requires_grad=True)
    vm_static = torch.empty(batch, 12, device=dev)
    tgt_static = torch.empty(batch * 3 * W * H, device=dev)
    views = _lib.Views(vm_static, intr[:batch].contiguous(), [W] * batch, [H] * batch, [0] * batch, [n] * batch)

    def load(k):
        ids = torch.as_tensor(synth.minibatch(k, n_views, batch), device=dev)
        vm = pose.apply_residual(noisy_vm[ids], dr[ids], dt[ids])
        with torch.no_grad():
            vm_static.copy_(vm)
            tgt_static.copy_(targets[ids].reshape(-1))
        return vm

    vm = load(0)
    from paper_2509_25191_gb300.tune import autotune
    choice, _ = autotune(g, views, tgt_static, tiles=SECONDARY_TILES, reps=3)
    tile = choice.tile
    step = GraphStep(g, views, tgt_static, tile=tile, batch=choice.batch)
    # Eq. 1 update state: Adam moments per group, a pool of exploration noise
    gp = [g.means, g.log_scales, g.quats, g.opacity_logits, g.sh]
    gg = [step.grads.means, step.grads.log_scales, step.grads.quats, step.grads.opacity_logits, step.grads.sh]
    lrs = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]
    mom = [(torch.zeros_like(p), torch.zeros_like(p)) for p in gp]
    noise = torch.randn(4, n, 3, device=dev, generator=torch.Generator(dev).manual_seed(11))
    pose_m = [(torch.zeros_like(dr), torch.zeros_like(dr)), (torch.zeros_like(dt), torch.zeros_like(dt))]

    last = {}

    def update(k):
        last["pose_grad_norm"] = float(torch.cat([dr.grad.reshape(-1), dt.grad.reshape(-1)]).norm())
        groups = [(p, gr, m, v, lr) for p, gr, (m, v), lr in zip(gp, gg, mom, lrs)]
        _lib.gs_sgld_adam_step(groups, k + 1, noise=noise[k % 4], noise_scale=1e-4, noise_group=0)
        lr_pose = pose.pose_lr(k)                       # Section 4.1: 1e-4 decayed exponentially to x0.1
        _lib.gs_sgld_adam_step([(dr.data, dr.grad, pose_m[0][0], pose_m[0][1], lr_pose),
                                (dt.data, dt.grad, pose_m[1][0], pose_m[1][1], lr_pose)], k + 1)
        dr.grad.zero_()
        dt.grad.zero_()

    for k in range(3):
        vm = load(k)
        step.replay()
        vm.backward(step.dviewmat)
        update(k)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for k in range(steps):
        vm = load(100 + k)
        step.replay()
        vm.backward(step.dviewmat)        # chain dL/d(R,t) to the 6D and translation residuals
        update(3 + k)
    b.record()
    torch.cuda.synchronize()
    if step.check():
        raise RuntimeError("capacity overflow during the dense step")
    ms = a.elapsed_time(b) / steps
    # where the rasterizer step's time goes (eager calls, per-stage events)
    sn = list(step.stages)
    sacc = np.zeros(len(sn))
    for _ in range(3):
        ev = []
        step.run(ev)
        torch.cuda.synchronize()
        sacc += [ev[i].elapsed_time(ev[i + 1]) for i in range(len(sn))]
    dense_stages = {k: round(float(v) / 3, 4) for k, v in zip(sn, sacc)}
    graph_ms = _time_replays(step, 10)
    dbytes = algorithmic_bytes(g.n, g.sh_degree, views.num_slots(), int(step.bins.counters[0].item()), views.pixels,
                               views.num_tiles(step.cfg))
    # the Eq. 1 update alone, against the HBM roofline (every element: read p, g, m, v; write p, m, v)
    a.record()
    for k in range(5):
        _lib.gs_sgld_adam_step([(p, gr, m, v, lr) for p, gr, (m, v), lr in zip(gp, gg, mom, lrs)], 100 + k,
                               noise=noise[k % 4], noise_scale=1e-4, noise_group=0)
    b.record()
    torch.cuda.synchronize()
    opt_ms = a.elapsed_time(b) / 5
    opt_bytes = 28 * sum(p.numel() for p in gp) + 12 * n
    peaks, _ = measured_peaks()
    px = batch * W * H
    opt = {"ms": round(opt_ms, 4), "algorithmic_bytes": opt_bytes,
           "achieved_gbs": round(opt_bytes / opt_ms / 1e6, 1),
           "frac_of_measured_hbm": round(opt_bytes / opt_ms / 1e6 / peaks["hbm_gbs"], 4)}
    return {"workload": "6M SH3 Gaussians, 300 jittered hemisphere views 1600x1066, minibatch 8, L1 vs targets, "
                        "backward to Gaussians and poses (6D + translation residuals), Eq. 1 SGLD/Adam update",
            "ms_per_step": round(ms, 3), "mpix_s": round(px / ms / 1e3, 2), "pixels_per_step": px,
            "rasterizer_graph_ms": round(graph_ms, 3), "rasterizer_stages_ms": dense_stages,
            "rasterizer_hbm_roofline": {"algorithmic_bytes": int(dbytes),
                                        "frac": round(dbytes / (graph_ms * 1e-3) / (measured_peaks()[0]["hbm_gbs"] * 1e9),
                                                      4)},
            "gaussian_order": "spatial (Morton) order, as the training loop keeps it",
            "sgld_adam_update": opt,
            "pose_grad_norm_last_step": round(last["pose_grad_norm"], 6),
            "tile": list(tile), "batch": list(choice.batch), "instances": int(step.bins.counters[0].item())}


def _rel_rot_err_deg(vm_a, vm_b, pairs):
    """Mean angle (degrees) between the relative rotations R_j R_i^T of two
    camera sets over the pairs (gauge-free pose error)."""
    Ra = vm_a[:, :9].reshape(-1, 3, 3).astype(np.float64)
    Rb = vm_b[:, :9].reshape(-1, 3, 3).astype(np.float64)
    i, j = pairs[:, 0], pairs[:, 1]
    A = Ra[j] @ np.transpose(Ra[i], (0, 2, 1))
    B = Rb[j] @ np.transpose(Rb[i], (0, 2, 1))
    c = (np.einsum("kab,kab->k", A, B) - 1.0) / 2.0
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))).mean())


def run_ga(dev, iterations=300, reps=50):
    """Camera global alignment (Section 3.3): 300 hemisphere cameras with
    jittered initial estimates (1 degree, 1 % translation, 2 % focal), pairs
    within 30 degrees, 4,096 matches per pair (0.5 px noise, 15 % outliers);
    Eq. 3 weights and the Eq. 4 learning rate from the initial distances,
    then 300 Adam iterations on 6D rotation, translation and log-focal
    residuals."""
    import torch

    from paper_2509_25191_gb300 import ga, synth
    tv, ti, iv, ii = synth.ga_cameras(0)
    vm0 = torch.as_tensor(iv, device=dev)
    intr0 = torch.as_tensor(ii, device=dev)
    pairs = ga.select_pairs(vm0, 30.0)
    pairs_h = pairs.cpu().numpy()
    M = synth.ga_matches(1, synth.ga_points(0), ti, tv, pairs_h, 1600, 1066)
    offs = torch.as_tensor(M.offsets, device=dev)
    mt = torch.as_tensor(M.matches, device=dev)
    G = ga.GlobalAlignment(intr0, vm0, pairs, offs, mt)
    intr, vm = G.cameras()
    for _ in range(3):
        G.loss_and_grads(intr, vm)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        G.loss_and_grads(intr, vm)
    b.record()
    torch.cuda.synchronize()
    k_ms = a.elapsed_time(b) / reps
    n_m, n_p = len(M.matches), len(pairs_h)
    nbytes = 20 * n_m + 64 * n_p          # match + weight per match; pair, offsets, partial sums per pair
    peaks, _ = measured_peaks()
    d0 = G.dist0.cpu().numpy()
    a.record()
    G.run(iterations)
    b.record()
    torch.cuda.synchronize()
    G.check()
    it_ms = a.elapsed_time(b) / iterations
    intr1, vm1 = G.cameras()
    d1 = torch.empty_like(G.dist0)
    from paper_2509_25191_gb300 import _lib
    _lib.gs_ga_epipolar(_lib.ga_problem(intr1.contiguous(), vm1.contiguous(), pairs, offs, mt), G.pair_sums,
                        G.loss, dist=d1)
    d1 = d1.cpu().numpy()
    inl = M.inlier
    return {"workload": "300 hemisphere cameras (jittered 1 deg / 1 % / focal 2 %), pairs within 30 deg, "
                        "4096 matches per pair with 15 % outliers, Eq. 2-4, 300 Adam iterations",
            "cameras": 300, "pairs": n_p, "matches": n_m, "median0_px": round(G.median0, 4), "lr": G.lr,
            "loss_and_grads_ms": round(k_ms, 4), "algorithmic_bytes": nbytes,
            "achieved_gbs": round(nbytes / k_ms / 1e6, 1),
            "frac_of_measured_hbm": round(nbytes / k_ms / 1e6 / peaks["hbm_gbs"], 4),
            "ms_per_iteration": round(it_ms, 4), "iterations": iterations,
            "rel_rot_err_deg": [round(_rel_rot_err_deg(tv, iv, pairs_h), 4),
                                round(_rel_rot_err_deg(tv, vm1.detach().cpu().numpy(), pairs_h), 4)],
            "inlier_median_px": [round(float(np.median(d0[inl])), 4), round(float(np.median(d1[inl])), 4)]}


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------

def oracle_step(sc, vw, fraction, seed, threads=1):
    """One oracle fwd + L1 + bwd + pose pass over a random pixel sample (all
    pixels if fraction >= 1), against the native arm's target image (uniform
    values, seed 1234); threads > 1 splits its projection and render passes
    over that many threads. Returns the number of pixels computed."""
    from oracle import oracle as O
    W, H = int(vw.width[0]), int(vw.height[0])
    rng = np.random.default_rng(seed)
    mask = None if fraction >= 1 else rng.random((H, W)) < fraction
    f = O.forward(sc, vw, masks=None if mask is None else [mask], threads=threads)
    target = np.random.default_rng(1234).uniform(0, 1, 3 * W * H).astype(np.float32).reshape(3, H, W)
    up = np.sign(f[0]["image"] - target) / (3.0 * W * H)          # the mean-L1 gradient
    if mask is not None:
        up[:, ~mask] = 0.0
    O.backward(sc, vw, f, [up], threads=threads)
    return W * H if mask is None else int(mask.sum())


def oracle_views():
    """The FP64 oracle (single thread) on one whole view of each
    configuration: projection, binning and render forward of every pixel,
    the mean-L1 gradient against a uniform target, render and projection
    backward and the pose gradient; per view, labelled, not extrapolated."""
    from paper_2509_25191_gb300 import synth
    out = {}
    cases = [("2,000 SH0 Gaussians, 128x128", lambda: synth.single_view_small()),
             ("1M clustered SH3, 1237x822", lambda: synth.single_view_1m(0)),
             ("500K clustered SH3, view 0 of the 16-view 979x546 orbit",
              lambda: (lambda sc, vw: (sc, vw.select([0])))(*synth.orbit_views(0, 500_000, 16, 979, 546))),
             ("uneven scenes: the 3M-Gaussian scene, its first view",
              lambda: _uneven_first_view()),
             ("6M SH3 dense scene, view 0 of minibatch 0 (1600x1066)",
              lambda: (lambda sc, tv, nv: (sc, nv.select(synth.minibatch(0, nv.n, 8)[:1])))(*synth.dense_hemisphere(0)))]
    for name, make in cases:
        sc, vw = make()
        t = time.perf_counter()
        px = oracle_step(sc, vw, 1.0, 7)
        out[name] = {"seconds_per_view": round(time.perf_counter() - t, 2), "pixels": px, "threads": 1}
    return out


def _uneven_first_view():
    from paper_2509_25191_gb300 import synth
    sc, vw = synth.uneven_scenes()
    v = int(np.argmax(vw.gauss_count))
    b, c = int(vw.gauss_begin[v]), int(vw.gauss_count[v])
    one = vw.select([v])
    one.gauss_begin[:] = 0
    return sc.subset(np.arange(b, b + c)), one


def cpu_baseline(sc, vw):
    """The FP64 oracle on the host: one full step threaded over all cores
    (the reported value) and one single-threaded, and the small workload."""
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    npx = oracle_step(sc, vw, 1.0, 7, threads=cores)
    dt = time.perf_counter() - t
    t = time.perf_counter()
    oracle_step(sc, vw, 1.0, 7)
    dt1 = time.perf_counter() - t
    out = {"value": round(npx / dt / 1e6, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"one full step: all {npx} pixels of the same workload, FP64 C oracle, projection and render "
                     f"passes threaded over {cores} host cores (binning single-threaded)",
           "seconds": round(dt, 2),
           "single_thread": {"seconds": round(dt1, 2), "mpix_s": round(npx / dt1 / 1e6, 6)}}
    # the small 2,000-Gaussian 128x128 case as well (full step, single thread)
    from paper_2509_25191_gb300 import synth
    ssc, svw = synth.single_view_small()
    for threads in (1, cores):
        t = time.perf_counter()
        reps = 0
        while time.perf_counter() - t < 1.0:
            spx = oracle_step(ssc, svw, 1.0, 7 + reps, threads=threads)
            reps += 1
        sdt = (time.perf_counter() - t) / reps
        out["small_case" if threads == 1 else "small_case_threaded"] = {
            "workload": "2,000 SH0 Gaussians, one 128x128 view", "threads": threads,
            "mpix_s": round(spx / sdt / 1e6, 6), "ms_per_step": round(sdt * 1e3, 3)}
    return out


_WORKER = {}


def _ref_worker_init(n):
    _WORKER["scene"] = workload(n)


def _ref_worker_step(job):
    fraction, seed = job
    sc, vw = _WORKER["scene"]
    return oracle_step(sc, vw, fraction, seed)


def run_reference(args, rank, world):
    """The oracle as it stands (single-threaded FP64 C), one step per worker
    process; steps run concurrently on the host cores (spawned pool)."""
    if rank != 0:
        return None
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    cores = max(1, min(os.cpu_count() or 1, args.steps))
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_ref_worker_init, initargs=(args.n,)) as pool:
        pool.map(_ref_worker_step, [(args.ref_fraction, 10_000 + w) for w in range(max(args.warmup, cores))])
        t = time.perf_counter()
        px = sum(pool.map(_ref_worker_step, [(args.ref_fraction, k) for k in range(args.steps)], chunksize=1))
        dt = time.perf_counter() - t
    val = px / dt / 1e6
    if args.ref_fraction >= 1.0:
        sample = (f"each step: the whole workload (projection, binning, render forward and backward of all 1237x822 "
                  f"pixels, projection backward and pose gradient of all {args.n} Gaussians); FP64 C oracle, "
                  f"single-threaded per step, {cores} steps at a time on {cores} host cores")
    else:
        sample = (f"each step: full projection, binning and projection backward of all {args.n} Gaussians, render "
                  f"forward+backward on a random {args.ref_fraction:.4f} of the 1237x822 pixels; FP64 C oracle, "
                  f"single-threaded per step, {cores} steps at a time on {cores} host cores")
    return {"metric": METRIC, "value": round(val, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"single view 1237x822, {args.n} clustered SH3 Gaussians (seed 0), fwd+L1+bwd+pose",
                       "gaussians": args.n, "views": 1, "pixels_per_step": 1237 * 822},
            "cpu_baseline": {"value": round(val, 6), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(val, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.only == "ga":
        import torch
        print(json.dumps(run_ga(torch.device("cuda", local_rank))), flush=True)
        return
    if args.only == "oracle_views":
        from oracle import oracle as O
        O.build()
        print(json.dumps({"oracle_per_view": oracle_views()}), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out, sc, vw = run_native(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(sc, vw)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
