"""Autotuners for the batched summary and for desummarisation.

The batched path: the size of its persistent grids (SMs x multiplier).  The
tuner times graph replays of the real batch for each candidate with CUDA
events, keeps the fastest, and caches the choice in a JSON file keyed by the
GPU and a coarse signature of the batch (rows, relations, tree depth, key
bits), so a later batch of the same shape skips the timing.

Desummarisation: the emit kernel's rows per thread, timed on a real window
of the query and cached by the GPU and the result's shape (tune_emit).

The summary: how the downward pass combines contributions to a child's down
message (GJ_OPT_DOWN_COMBINE) for a join tree, or how the 3-cycle finds its
group triples (GJ_OPT_TRIANGLE_INTERSECT), timed on the query's own
gj_summarize and cached by the GPU and the query's shape (tune_summary).
"""
from __future__ import annotations

import json
import math
import os

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
CANDIDATES = (1, 2, 4, 8, 16)


def _load_cache(path, use):
    """The cache file's entries ({} when unused, missing or unreadable)."""
    if use and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
            return cache if isinstance(cache, dict) else {}
        except (OSError, ValueError):
            return {}
    return {}


def _store_cache(path, cache):
    """Writes the cache through a temporary file renamed over the old one, so
    a reader never sees a partial file."""
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)


def signature(batch, gpu_name: str) -> str:
    rows = 0 if batch.n_rows <= 0 else int(round(math.log2(batch.n_rows)))
    return f"{gpu_name}|rows2^{rows}|rel{batch.n_relations}|lv{batch.levels}|bits{batch.key_bits}"


def tune_batch(batch, candidates=CANDIDATES, reps: int = 3, cache_path: str = DEFAULT_CACHE,
               use_cache: bool = True) -> dict:
    import torch
    gpu = torch.cuda.get_device_name(batch.ctx.device)
    key = signature(batch, gpu)
    cache = _load_cache(cache_path, use_cache)
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
        _store_cache(cache_path, cache)
    return dict(entry, cached=False)


# ---------------------------------------------------------------- emit
# The desummarise emit kernel writes RPT consecutive rows per thread (2, 4 or
# 8): more rows per thread mean fewer block lookups per row, fewer mean more
# threads in flight.  Which is faster depends on the GPU and on the result's
# shape (relations, and how many rows a key path's block holds), so the
# tuner times one real window per choice and caches the best.
EMIT_RPT = (2, 4, 8)


def emit_signature(query, gpu_name: str, window: int) -> str:
    rows_per_block = 0
    try:
        groups = max(1, min(query.n_groups))
        rows_per_block = int(round(math.log2(max(1, (query.total or 1) / groups))))
    except (TypeError, ValueError):
        pass
    return f"{gpu_name}|emit|rel{query.n_rel}|cols{len(query.col_width)}|rpb2^{rows_per_block}|win2^{int(math.log2(window))}"


def tune_emit(ctx, query, window: int = 1 << 24, reps: int = 3, cache_path: str = DEFAULT_CACHE,
              use_cache: bool = True) -> dict:
    """Times gj_desummarize of the query's first `window` rows for every
    rows-per-thread choice; leaves the fastest set on the context (the
    option is read at each launch) and returns it with the timings."""
    import torch
    from . import gj
    gpu = torch.cuda.get_device_name(ctx.device)
    total = query.total
    if not total:
        return {"rpt": 4, "skipped": "empty result"}
    n = min(window, total)
    key = emit_signature(query, gpu, n)
    cache = _load_cache(cache_path, use_cache)
    if use_cache and key in cache:
        ctx.set_option(gj.GJ_OPT_EMIT_ROWS_PER_THREAD, int(cache[key]["rpt"]))
        return dict(cache[key], cached=True)
    out = query.alloc_columns(n)
    stream = ctx.stream
    times = {}
    for rpt in EMIT_RPT:
        ctx.set_option(gj.GJ_OPT_EMIT_ROWS_PER_THREAD, rpt)
        query.desummarize(0, n, out=out)      # warm-up
        stream.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            query.desummarize(0, n, out=out)
        t1.record(stream)
        t1.synchronize()
        times[rpt] = t0.elapsed_time(t1) / reps
    best = min(times, key=times.get)
    ctx.set_option(gj.GJ_OPT_EMIT_ROWS_PER_THREAD, best)
    entry = {"rpt": best, "ms": times[best], "candidates_ms": {str(k): v for k, v in times.items()}}
    if use_cache:
        cache[key] = entry
        _store_cache(cache_path, cache)
    return dict(entry, cached=False)


# ---------------------------------------------------------------- summary
def summary_signature(query, gpu_name: str, kind: str) -> str:
    groups = [max(1, g) for g in query.n_groups]
    g2 = "-".join(str(int(round(math.log2(g)))) for g in groups)
    tree = "-".join(str(p) for p in query.parent)
    return f"{gpu_name}|summary|{kind}|rel{query.n_rel}|groups2^{g2}|parents{tree}"


def tune_summary(ctx, query, triangle: bool = False, reps: int = 3, cache_path: str = DEFAULT_CACHE,
                 use_cache: bool = True) -> dict:
    """Times gj_summarize of the query for every choice of the summary's
    option -- GJ_OPT_TRIANGLE_INTERSECT (1 sorted lists, 2 bitmaps) for the
    3-cycle, GJ_OPT_DOWN_COMBINE (0 by key order, 1 never, 2 always)
    otherwise -- and leaves the fastest set on the context.  Every choice
    gives the same summary; the timings and the choice are returned."""
    import torch
    from . import gj
    opt, cands, name = ((gj.GJ_OPT_TRIANGLE_INTERSECT, (1, 2), "triangle_intersect") if triangle
                        else (gj.GJ_OPT_DOWN_COMBINE, (0, 1, 2), "down_combine"))
    gpu = torch.cuda.get_device_name(ctx.device)
    key = summary_signature(query, gpu, name)
    cache = _load_cache(cache_path, use_cache)
    if use_cache and key in cache:
        ctx.set_option(opt, int(cache[key][name]))
        return dict(cache[key], cached=True)
    stream = ctx.stream
    times, totals = {}, {}
    for v in cands:
        ctx.set_option(opt, v)
        totals[v] = _summarize_or_sat(query, gj)    # warm-up, and the result to compare
        stream.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            _summarize_or_sat(query, gj)
        t1.record(stream)
        t1.synchronize()
        times[v] = t0.elapsed_time(t1) / reps
    if len(set(totals.values())) != 1:
        raise RuntimeError(f"summary options disagree on |Q|: {totals}")
    best = min(times, key=times.get)
    ctx.set_option(opt, best)
    entry = {name: best, "ms": times[best], "candidates_ms": {str(k): v for k, v in times.items()}}
    if use_cache:
        cache[key] = entry
        _store_cache(cache_path, cache)
    return dict(entry, cached=False)


def _summarize_or_sat(query, gj):
    try:
        return query.summarize()
    except gj.GJError as e:
        if e.status != gj.GJ_ERR_OVERFLOW:
            raise
        return gj.SAT
