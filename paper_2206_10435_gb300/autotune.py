"""Autotuner for the batched summary.

The batched path has one tunable that matters on a given GPU and batch
shape: the size of its persistent grids (SMs x multiplier).  The tuner times
graph replays of the real batch for each candidate with CUDA events, keeps
the fastest, and caches the choice in a JSON file keyed by the GPU and a
coarse signature of the batch (rows, relations, tree depth, key bits), so a
later batch of the same shape skips the timing.
"""
from __future__ import annotations

import json
import math
import os

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
CANDIDATES = (1, 2, 4, 8, 16)


def signature(batch, gpu_name: str) -> str:
    rows = 0 if batch.n_rows <= 0 else int(round(math.log2(batch.n_rows)))
    return f"{gpu_name}|rows2^{rows}|rel{batch.n_relations}|lv{batch.levels}|bits{batch.key_bits}"


def tune_batch(batch, candidates=CANDIDATES, reps: int = 3, cache_path: str = DEFAULT_CACHE,
               use_cache: bool = True) -> dict:
    import torch
    gpu = torch.cuda.get_device_name(batch.ctx.device)
    key = signature(batch, gpu)
    cache = {}
    if use_cache and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        batch.set_grid_mult(int(cache[key]["grid_mult"]))
        return dict(cache[key], cached=True)
    stream = batch.ctx.stream
    times = {}
    for m in candidates:
        batch.set_grid_mult(m)
        batch.run(use_graph=True)            # capture + first launch
        stream.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            batch.run(use_graph=True)
        t1.record(stream)
        t1.synchronize()
        times[m] = t0.elapsed_time(t1) / reps
    best = min(times, key=times.get)
    batch.set_grid_mult(best)
    entry = {"grid_mult": best, "ms": times[best], "candidates_ms": {str(k): v for k, v in times.items()}}
    if use_cache:
        cache[key] = entry
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".{os.getpid()}.tmp"
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, cache_path)
    return dict(entry, cached=False)
