"""Autotuner for the launch choices exposed by occ_tuning.

For a workload key (image size, pattern, K, formats, effect, estimator) it times each
candidate configuration on the caller's own buffers with CUDA events, keeps the fastest,
and stores it in a JSON cache so later runs apply it without measuring:

  * reuse of window patterns (box / offsets): TMA-staged tile kernel with 4, 8 or 16
    receiver rows per tile, or the per-receiver kernel;
  * reuse of group patterns: the group kernel's L2 prefetch (none, G-buffer and records);
  * the step-1 trace: one CTA per 16 x 8 tile, or persistent CTAs taking rays from a
    counter with a refill threshold of 8, 16 or 24 idle lanes, all or half of the CTAs that
    fit, and the rays handed out by tiles row-major or by 8 x 8-tile blocks in Morton order;
  * persistent batched kernels: CTAs per SM (1, 2, 4, 8 or all that fit);
  * the G-buffer layout: row-major, or 8 x 8-pixel tiles in Morton order (a tiled copy made
    once by occ_tile_gbuffer), timed over a whole frame (step-1 trace + reuse).

Cache: $OCC_TUNE_CACHE, else ~/.cache/occreuse/tuning.json.
"""
from __future__ import annotations

import json
import os
import threading

from . import occ as O

_LOCK = threading.Lock()

REUSE_CANDIDATES = [
    {"reuse_tile_rows": 16, "reuse_window_path": 1},
    {"reuse_tile_rows": 16, "reuse_window_path": 3},
    {"reuse_tile_rows": 8, "reuse_window_path": 1},
    {"reuse_tile_rows": 4, "reuse_window_path": 1},
    {"reuse_tile_rows": 0, "reuse_window_path": 2},
]
GROUP_CANDIDATES = [{"group_prefetch": c} for c in (1, 2, 3)]
TRACE_CANDIDATES = [{"trace_path": 1}] + [
    {"trace_path": 2, "trace_refill": r, "trace_ctas_per_sm": c, "trace_order": o}
    for r in (8, 16, 24) for c in (0, 4) for o in (1, 2)]
BATCH_CANDIDATES = [{"batch_ctas_per_sm": n} for n in (0, 1, 2, 4, 8)]


def cache_path() -> str:
    return os.environ.get("OCC_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "occreuse",
                                       "tuning.json"))


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def reuse_key(gb: O.GBuffer, rec: O.Occluders, pattern: O.Pattern, estimator: int,
              effect: int) -> str:
    return (f"reuse/{gb.W}x{gb.H}/pat{pattern.kind}:{pattern.gw}x{pattern.gh}/K{pattern.K}/"
            f"gb{int(gb.packed)}/rec{int(rec.packed)}/eff{effect}/est{estimator}")


def trace_key(gb: O.GBuffer, rec: O.Occluders, bvh: O.BVH, effect: int) -> str:
    return (f"trace/{gb.W}x{gb.H}/gb{int(gb.packed)}/rec{int(rec.packed)}/eff{effect}/"
            f"tris{bvh.stats['num_tris']}")


def layout_key(gb: O.GBuffer, rec: O.Occluders, pattern: O.Pattern, estimator: int,
               effect: int) -> str:
    return (f"layout/{gb.W}x{gb.H}/pat{pattern.kind}:{pattern.gw}x{pattern.gh}/K{pattern.K}/"
            f"gb{int(gb.packed)}/rec{int(rec.packed)}/eff{effect}/est{estimator}")


def batch_key(views: list) -> str:
    px = sum(v.gb.W * v.gb.H for v in views)
    kinds = sorted({(v.effect, v.estimator, v.pattern.K) for v in views})
    return f"batch/{len(views)}views/{px}px/{kinds}"


def _time(fn, iters: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]   # median, ms


def _apply(ctx: O.Context, cfg: dict) -> None:
    base = O.occ_get_tuning(ctx)
    base.update(cfg)
    O.occ_set_tuning(ctx, **base)


def tune_reuse(ctx: O.Context, gb: O.GBuffer, rec: O.Occluders, pattern: O.Pattern,
               estimator: int, out, bvh=None, iters: int = 15, use_cache: bool = True) -> dict:
    """Picks the window-reuse configuration for this workload and applies it to ctx."""
    key = reuse_key(gb, rec, pattern, estimator, rec.meta.effect)
    with _LOCK:
        cache = load_cache() if use_cache else {}
    if key in cache:
        _apply(ctx, cache[key]["best"])
        return cache[key]
    fn = O.occ_reuse_ao if rec.meta.effect == O.OCC_EFFECT_AO else O.occ_reuse_shadow
    timings = []
    cands = REUSE_CANDIDATES if pattern.kind != O.OCC_PAT_GROUP else GROUP_CANDIDATES
    for cfg in cands:
        _apply(ctx, cfg)
        ms = _time(lambda: fn(ctx, gb, rec, pattern, pattern.K, estimator, bvh=bvh, out=out), iters)
        timings.append({"config": cfg, "ms": ms})
    best = min(timings, key=lambda t: t["ms"])
    entry = {"best": best["config"], "timings": timings}
    _apply(ctx, best["config"])
    with _LOCK:
        cache = load_cache()
        cache[key] = entry
        save_cache(cache)
    return entry


def tune_trace(ctx: O.Context, gb: O.GBuffer, bvh: O.BVH, effect: int, rec: O.Occluders,
               radius: float = 0.0, light=None, iters: int = 15, use_cache: bool = True) -> dict:
    """Picks the step-1 trace launch (kernel, refill threshold, CTAs per SM) for this
    workload, timing it into the caller's record buffer, and applies it to ctx."""
    key = trace_key(gb, rec, bvh, effect)
    with _LOCK:
        cache = load_cache() if use_cache else {}
    if key in cache:
        _apply(ctx, cache[key]["best"])
        return cache[key]

    def run():
        if effect == O.OCC_EFFECT_AO:
            O.occ_trace_ao(ctx, gb, bvh, radius, 1, 0, out=rec)
        else:
            O.occ_trace_shadow(ctx, gb, bvh, light, 1, 0, out=rec)

    timings = []
    for cfg in TRACE_CANDIDATES:
        full = {"trace_path": 0, "trace_refill": 0, "trace_ctas_per_sm": 0, "trace_order": 0}
        full.update(cfg)
        _apply(ctx, full)
        timings.append({"config": full, "ms": _time(run, iters)})
    best = min(timings, key=lambda t: t["ms"])
    entry = {"best": best["config"], "timings": timings}
    _apply(ctx, best["config"])
    with _LOCK:
        cache = load_cache()
        cache[key] = entry
        save_cache(cache)
    return entry


def tune_batch(ctx: O.Context, bvh: O.BVH, views: list, iters: int = 10,
               use_cache: bool = True) -> dict:
    """Picks the CTAs-per-SM of the persistent batched kernels for this view mix."""
    key = batch_key(views)
    with _LOCK:
        cache = load_cache() if use_cache else {}
    if key in cache:
        _apply(ctx, cache[key]["best"])
        return cache[key]
    timings = []
    for cfg in BATCH_CANDIDATES:
        _apply(ctx, cfg)
        ms = _time(lambda: O.occ_frame_batch(ctx, bvh, views), iters)
        timings.append({"config": cfg, "ms": ms})
    best = min(timings, key=lambda t: t["ms"])
    entry = {"best": best["config"], "timings": timings}
    _apply(ctx, best["config"])
    with _LOCK:
        cache = load_cache()
        cache[key] = entry
        save_cache(cache)
    return entry


LAYOUT_CANDIDATES = ("linear", "tiled")


def tune_layout(ctx: O.Context, gb: O.GBuffer, bvh: O.BVH, effect: int, pattern: O.Pattern,
                estimator: int, rec: O.Occluders, out, radius: float = 0.0, light=None,
                iters: int = 10, use_cache: bool = True) -> dict:
    """Picks the G-buffer layout for this workload: the caller's row-major G-buffer or a
    tiled copy of it (made once, outside the timing), each timed over a frame (step-1 trace
    into `rec`, then reuse into `out`).  Returns the cache entry plus "gbuffer": the G-buffer
    to use (the tiled copy when it won)."""
    key = layout_key(gb, rec, pattern, estimator, effect)
    with _LOCK:
        cache = load_cache() if use_cache else {}
    if key in cache:
        entry = dict(cache[key])
        entry["gbuffer"] = (O.occ_tile_gbuffer(ctx, gb)
                            if entry["best"]["gbuffer_layout"] == "tiled" else gb)
        return entry
    tiled = O.occ_tile_gbuffer(ctx, gb)
    reuse = O.occ_reuse_ao if effect == O.OCC_EFFECT_AO else O.occ_reuse_shadow
    traces = estimator in (O.OCC_EST_UNBIASED, O.OCC_EST_LIGHT_UNBIASED)

    def frame(g):
        if effect == O.OCC_EFFECT_AO:
            O.occ_trace_ao(ctx, g, bvh, radius, 1, 0, out=rec)
        else:
            O.occ_trace_shadow(ctx, g, bvh, light, 1, 0, out=rec)
        reuse(ctx, g, rec, pattern, pattern.K, estimator, bvh=bvh if traces else None, out=out)

    timings = []
    for name, g in zip(LAYOUT_CANDIDATES, (gb, tiled)):
        timings.append({"config": {"gbuffer_layout": name}, "ms": _time(lambda: frame(g), iters)})
    best = min(timings, key=lambda t: t["ms"])
    entry = {"best": best["config"], "timings": timings}
    with _LOCK:
        cache = load_cache()
        cache[key] = entry
        save_cache(cache)
    entry = dict(entry)
    entry["gbuffer"] = tiled if best["config"]["gbuffer_layout"] == "tiled" else gb
    return entry
