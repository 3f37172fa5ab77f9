"""Autotuner for the rasterizer's launch shape.

The tile shape sets both the binning granularity (instances per Gaussian)
and the raster kernels' block shape, and the best choice depends on the
scene (Gaussian footprints), the resolution and the number of views. The
tuner times the whole captured training step (GraphStep) for each candidate
tile shape on the caller's own inputs and keeps the fastest. The shared
memory batch is tied to the tile (per batch the forward stages one Gaussian
per pixel of the tile, the backward one per thread, i.e. per two pixels), so
choosing the tile chooses the batch. Results are cached in a JSON file
keyed by GPU name and a coarse workload signature (Gaussian count, views,
pixels, SH degree), so a training run pays for tuning once.
"""
from __future__ import annotations

import json
import math
import os

import torch

from ._lib import Gaussians, Views
from .step import GraphStep

CANDIDATES = ((16, 16), (32, 8), (16, 8), (8, 8), (32, 16), (32, 32))


def signature(g: Gaussians, views: Views) -> str:
    dev = torch.cuda.get_device_name(g.means.device)
    n_b = int(round(math.log2(max(1, g.n))))
    px_b = int(round(math.log2(max(1, views.pixels))))
    return f"{dev}|n2^{n_b}|v{views.n}|px2^{px_b}|sh{g.sh_degree}"


def _load(path):
    if path and os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}
    return {}


def autotune(g: Gaussians, views: Views, target, candidates=CANDIDATES, reps=10, cache_path=None, force=False):
    """Return (best_tile, {tile: ms_per_step}) for one step on these inputs."""
    key = signature(g, views)
    cache = _load(cache_path)
    if not force and key in cache:
        e = cache[key]
        return tuple(e["tile"]), {tuple(map(int, k.split("x"))): v for k, v in e["ms"].items()}
    def time_step(step, n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            step.replay()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    # pass 1: every candidate once; pass 2: the two fastest, re-timed in
    # alternation (median of three) so that clock ramp-up, the order of the
    # candidates and a single outlying measurement do not decide between
    # near-equal shapes
    times = {}
    for tile in candidates:
        step = GraphStep(g, views, target, tile=tile)
        for _ in range(3):
            step.replay()
        torch.cuda.synchronize()
        t = time_step(step, reps)
        if step.check():          # capacity grew: rerun this candidate once
            t = time_step(step, reps)
        times[tuple(tile)] = t
        del step
        torch.cuda.empty_cache()
    finalists = sorted(times, key=times.get)[:2]
    if len(finalists) > 1:
        steps = {t: GraphStep(g, views, target, tile=t) for t in finalists}
        for st in steps.values():
            for _ in range(3):
                st.replay()
        torch.cuda.synchronize()
        again = {t: [] for t in finalists}
        for _ in range(3):
            for t, st in steps.items():
                again[t].append(time_step(st, 2 * reps))
        for t in finalists:
            times[t] = sorted(again[t])[1]
        del steps
        torch.cuda.empty_cache()
    best = min(times, key=times.get)
    if cache_path:
        cache[key] = {"tile": list(best), "ms": {f"{t[0]}x{t[1]}": v for t, v in times.items()}}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return best, times
