"""Autotuner for the rasterizer's launch shape: tile size and shared-memory
batch.

The tile shape sets both the binning granularity (instances per Gaussian)
and the raster kernels' block shape; the batch sets how many Gaussians each
thread stages per shared-memory batch in the forward and in the backward
(more per batch: fewer block barriers and tile-list reads per Gaussian, but
more shared memory and so fewer resident blocks). The best pair depends on
the scene (Gaussian footprints, depth complexity), the resolution and the
number of views. The tuner times the whole captured training step
(GraphStep) on the caller's own inputs:

  1. every tile shape at the default batch (2 forward, 1 backward);
  2. every other batch at the two fastest tiles;
  3. the two fastest (tile, batch) pairs again, three times in alternation,
     keeping the median, so that clock ramp-up, candidate order and one
     outlying measurement do not decide between near-equal choices.

Results are cached in a JSON file keyed by GPU name and a coarse workload
signature (Gaussian count, views, pixels, SH degree), so a training run pays
for tuning once. Every candidate renders the same image bit for bit (the
per-pixel arithmetic and the per-pixel order of Gaussians do not depend on
the launch shape), so the choice changes only the time.
"""
from __future__ import annotations

import json
import math
import os
from typing import NamedTuple

import torch

from ._lib import Gaussians, Views
from .step import GraphStep

TILES = ((16, 16), (32, 8), (16, 8), (8, 8), (32, 16), (32, 32))
DEFAULT_BATCH = (2, 1)
BATCHES = ((2, 1), (1, 1), (4, 1), (2, 2), (1, 2))   # (forward, backward) Gaussians per thread and batch


class Choice(NamedTuple):
    tile: tuple
    batch: tuple


def key_str(c: Choice) -> str:
    return f"{c.tile[0]}x{c.tile[1]}/{c.batch[0]}.{c.batch[1]}"


def parse_key(s: str) -> Choice:
    t, b = s.split("/")
    return Choice(tuple(map(int, t.split("x"))), tuple(map(int, b.split("."))))


def candidates(tiles=TILES, batches=BATCHES):
    """Every (tile, batch) pair the tuner may choose from."""
    return [Choice(tuple(t), tuple(b)) for t in tiles for b in batches]


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


def _time_step(step, n):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(n):
        step.replay()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / n


def autotune(g: Gaussians, views: Views, target, tiles=TILES, batches=BATCHES, reps=10, cache_path=None,
             force=False):
    """Return (Choice(tile, batch), {Choice: ms_per_step}) for one training
    step on these inputs."""
    key = signature(g, views)
    cache = _load(cache_path)
    if not force and key in cache:
        e = cache[key]
        return parse_key(e["best"]), {parse_key(k): v for k, v in e["ms"].items()}

    times = {}

    def measure(c: Choice):
        step = GraphStep(g, views, target, tile=c.tile, batch=c.batch)
        for _ in range(3):
            step.replay()
        torch.cuda.synchronize()
        t = _time_step(step, reps)
        if step.check():          # capacity grew: rerun this candidate once
            t = _time_step(step, reps)
        times[c] = t
        del step
        torch.cuda.empty_cache()

    default = tuple(batches[0]) if DEFAULT_BATCH not in [tuple(b) for b in batches] else DEFAULT_BATCH
    for t in tiles:                                   # 1. tiles at the default batch
        measure(Choice(tuple(t), default))
    best_tiles = sorted(times, key=times.get)[:2]
    for c in best_tiles:                              # 2. batches at the two fastest tiles
        for b in batches:
            if tuple(b) != default:
                measure(Choice(c.tile, tuple(b)))
    finalists = sorted(times, key=times.get)[:2]
    if len(finalists) > 1:                            # 3. the two fastest, in alternation
        steps = {c: GraphStep(g, views, target, tile=c.tile, batch=c.batch) for c in finalists}
        for st in steps.values():
            for _ in range(3):
                st.replay()
        torch.cuda.synchronize()
        again = {c: [] for c in finalists}
        for _ in range(3):
            for c, st in steps.items():
                again[c].append(_time_step(st, 2 * reps))
        for c in finalists:
            times[c] = sorted(again[c])[1]
        del steps
        torch.cuda.empty_cache()
    best = min(times, key=times.get)
    if cache_path:
        cache[key] = {"best": key_str(best), "ms": {key_str(c): v for c, v in times.items()}}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return best, times
