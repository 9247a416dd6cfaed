"""Image-quality harness: equal-time RelMSE of the estimators against a high-spp reference.

Follows the paper's evaluation (Sec. 5): the reference is the no-reuse estimator averaged
over many samples per pixel; each method runs as many 1-spp frames as fit a time budget at
the measured cost of one frame (trace + reuse), and its average is scored by

    RelMSE = mean over valid pixels of (est - ref)^2 / (ref^2 + eps),  eps = 1e-3,

reported beside its ratio to the no-reuse baseline at the same budget.  Methods: NOREUSE
(no reuse), the averaging filter over the shared group (Filter(N) for AO, Light(N) for
shadows: light-sample reuse without validation reduces to it), and biased occlusion-point
reuse Occ(N) on shared groups (N = 2, 4, 8 as 2x1, 2x2, 4x2 blocks) or window patterns.
Estimates are never clamped.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import occ as O

RELMSE_EPS = 1e-3
REF_SAMPLE_BASE = 0          # reference uses sample indices [0, spp)
EST_SAMPLE_BASE = 1 << 20    # estimates use indices from here: independent of the reference


def relmse(est: np.ndarray, ref: np.ndarray, valid: np.ndarray, eps: float = RELMSE_EPS) -> float:
    e = est.astype(np.float64)[valid] - ref.astype(np.float64)[valid]
    return float(np.mean(e * e / (ref.astype(np.float64)[valid] ** 2 + eps)))


def region_errors(est: np.ndarray, ref: np.ndarray, valid: np.ndarray,
                  eps: float = RELMSE_EPS) -> dict:
    """Errors by region of the reference: umbra (reference 0: every reference sample blocked),
    penumbra, lit (reference 1).  Per region: pixel count, MSE, share of the image's summed
    relative squared error, and mean error."""
    r = ref.astype(np.float64)[valid]
    e = est.astype(np.float64)[valid] - r
    rel = e * e / (r * r + eps)
    out = {}
    for name, m in (("umbra", r == 0.0), ("penumbra", (r > 0.0) & (r < 1.0)), ("lit", r == 1.0)):
        n = int(m.sum())
        out[name] = {"pixels": n, "mse": float(np.mean(e[m] * e[m])) if n else 0.0,
                     "relmse_share": float(rel[m].sum() / max(rel.sum(), 1e-300)),
                     "bias": float(np.mean(e[m])) if n else 0.0}
    return out


def _trace(ctx, gb, bvh, effect, radius, light, seed, sample, rec, stream=None):
    if effect == O.OCC_EFFECT_AO:
        return O.occ_trace_ao(ctx, gb, bvh, radius, seed, sample, out=rec, stream=stream)
    return O.occ_trace_shadow(ctx, gb, bvh, light, seed, sample, out=rec, stream=stream)


def _reuse(ctx, gb, rec, effect, pattern, estimator, bvh, out, stream=None):
    fn = O.occ_reuse_ao if effect == O.OCC_EFFECT_AO else O.occ_reuse_shadow
    traces = estimator in (O.OCC_EST_UNBIASED, O.OCC_EST_LIGHT_UNBIASED)
    return fn(ctx, gb, rec, pattern, pattern.K, estimator, bvh=bvh if traces else None, out=out,
              stream=stream)


def reference(ctx, gb, bvh, effect, radius=0.5, light=None, spp=4096, seed=1) -> np.ndarray:
    """Mean of `spp` no-reuse frames (sample indices 0 .. spp-1)."""
    dev = gb.pos4.device
    rec = O.Occluders.empty(gb.H, gb.W, dev, packed=gb.packed)
    out = torch.empty((gb.H, gb.W), dtype=torch.float32, device=dev)
    acc = torch.zeros((gb.H, gb.W), dtype=torch.float64, device=dev)
    one = O.Pattern.group(1, 1)
    for s in range(spp):
        _trace(ctx, gb, bvh, effect, radius, light, seed, REF_SAMPLE_BASE + s, rec)
        _reuse(ctx, gb, rec, effect, one, O.OCC_EST_NOREUSE, None, out)
        acc += out
    ctx.sync()
    return (acc / spp).cpu().numpy()


def frame_ms(ctx, gb, bvh, effect, pattern, estimator, radius=0.5, light=None, iters=20) -> float:
    """Mean time of one 1-spp frame (trace + reuse), CUDA events on the current stream."""
    dev = gb.pos4.device
    rec = O.Occluders.empty(gb.H, gb.W, dev, packed=gb.packed)
    out = torch.empty((gb.H, gb.W), dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream()
    for i in range(3):
        _trace(ctx, gb, bvh, effect, radius, light, 1, i, rec, st)
        _reuse(ctx, gb, rec, effect, pattern, estimator, bvh, out, st)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    for i in range(iters):
        _trace(ctx, gb, bvh, effect, radius, light, 1, i, rec, st)
        _reuse(ctx, gb, rec, effect, pattern, estimator, bvh, out, st)
    b.record(st)
    b.synchronize()
    ctx.sync()
    return a.elapsed_time(b) / iters


def estimate(ctx, gb, bvh, effect, pattern, estimator, frames, radius=0.5, light=None,
             seed=1) -> np.ndarray:
    """Mean of `frames` 1-spp estimates (independent of the reference's samples)."""
    dev = gb.pos4.device
    rec = O.Occluders.empty(gb.H, gb.W, dev, packed=gb.packed)
    out = torch.empty((gb.H, gb.W), dtype=torch.float32, device=dev)
    acc = torch.zeros((gb.H, gb.W), dtype=torch.float64, device=dev)
    for m in range(frames):
        _trace(ctx, gb, bvh, effect, radius, light, seed, EST_SAMPLE_BASE + m, rec)
        _reuse(ctx, gb, rec, effect, pattern, estimator, bvh, out)
        acc += out
    ctx.sync()
    return (acc / frames).cpu().numpy()


def methods(effect) -> list:
    """(name, pattern, estimator) of the compared methods."""
    avg = "Filter(8)" if effect == O.OCC_EFFECT_AO else "Light(8)"
    return [("NoReuse", O.Pattern.group(1, 1), O.OCC_EST_NOREUSE),
            (avg, O.Pattern.group(4, 2), O.OCC_EST_BOXMEAN),
            ("Occ(2)", O.Pattern.group(2, 1), O.OCC_EST_BIASED),
            ("Occ(4)", O.Pattern.group(2, 2), O.OCC_EST_BIASED),
            ("Occ(8)", O.Pattern.group(4, 2), O.OCC_EST_BIASED)]


def equal_time(ctx, gb, bvh, effect, budget_ms, ref, radius=0.5, light=None, extra=()) -> dict:
    """RelMSE of every method at `budget_ms` per image (frames = floor(budget / frame time),
    at least 1), and its ratio to NoReuse."""
    valid = gb.pos4[..., 3].cpu().numpy() != 0 if not gb.packed else \
        gb.pos4[..., 3].contiguous().view(torch.int32).cpu().numpy() != np.int32(-2147450880)
    rows = {}
    for name, pat, est in list(methods(effect)) + list(extra):
        t = frame_ms(ctx, gb, bvh, effect, pat, est, radius, light)
        frames = max(1, int(math.floor(budget_ms / t)))
        img = estimate(ctx, gb, bvh, effect, pat, est, frames, radius, light)
        e = img[valid].astype(np.float64) - ref[valid]
        rows[name] = {"frame_ms": t, "frames": frames, "relmse": relmse(img, ref, valid),
                      "mse": float(np.mean(e * e)), "bias": float(np.mean(e)),
                      "bins": region_errors(img, ref, valid)}
    base = rows["NoReuse"]["relmse"]
    for r in rows.values():
        r["ratio_to_noreuse"] = r["relmse"] / base if base > 0 else float("nan")
    return rows
