"""Comparison helpers shared by the GPU parity tests.

Tolerances (FP32 path against the FP64 oracle on identical inputs):
  * triangle ids bit-exact, except rays whose oracle margin (distance of a decision
    from its threshold: barycentric edge, t interval, tie) is below TRACE_MARGIN;
    such disagreements are listed and may not exceed DISAGREE_FRAC of the pixels
    (at least one pixel is allowed on small images);
  * hit distance error <= max(T_RTOL * t, T_ATOL * scale) + DIR_ERR * t / |cos i|, where
    scale = 1 + max|coordinate| (a hit near the ray origin carries the absolute rounding
    of the coordinates) and i is the incidence angle of the ray on the hit triangle (the
    FP32 ray direction differs from the FP64 one by ~DIR_ERR, which a grazing hit turns
    into a distance error); hit point error <= POS_ATOL * scale plus the same grazing term,
    normal error <= NRM_ATOL;
  * per-pixel AO / visibility <= OUT_ATOL absolute, except pixels whose reuse margin
    (support tests and validation rays) is below REUSE_MARGIN, listed likewise.
"""
import math

import numpy as np

TRACE_MARGIN = 1e-4
REUSE_MARGIN = 1e-4
DISAGREE_FRAC = 1e-4
T_RTOL = 1e-5
T_ATOL = 2.0 ** -20
DIR_ERR = 1e-6
POS_ATOL = 1e-5
NRM_ATOL = 2e-6
OUT_ATOL = 1e-5


def budget(n_pixels: int) -> int:
    return max(1, math.ceil(DISAGREE_FRAC * n_pixels))


def gpu_records(occ) -> tuple:
    """(rec0, rec1, tri) as NumPy from an Occluders object."""
    d = occ.data.cpu().numpy()
    tri = d[0, ..., 3].copy().view(np.int32)
    return d[0], d[1], tri


def to_f32_records(orec: np.ndarray) -> tuple:
    """Oracle FP64 records -> the FP32 record planes of the C ABI."""
    H, W = orec.shape[:2]
    r0 = np.zeros((H, W, 4), dtype=np.float32)
    r1 = np.zeros((H, W, 4), dtype=np.float32)
    r0[..., :3] = orec[..., :3]
    r0[..., 3] = orec[..., 7].astype(np.int32).view(np.float32)
    r1[..., :3] = orec[..., 3:6]
    r1[..., 3] = orec[..., 6]
    return r0, r1


def widen_records(r0: np.ndarray, r1: np.ndarray) -> np.ndarray:
    """FP32 record planes -> the oracle's FP64 layout (exact widening)."""
    H, W = r0.shape[:2]
    rec = np.zeros((H, W, 8))
    rec[..., :3] = r0[..., :3]
    rec[..., 3:6] = r1[..., :3]
    rec[..., 6] = r1[..., 3]
    rec[..., 7] = r0[..., 3].copy().view(np.int32)
    return rec


def _cos_incidence(orec: np.ndarray, pos4: np.ndarray, sel: np.ndarray) -> np.ndarray:
    """Cosine between each hit's ray (receiver -> hit point) and the hit normal."""
    w = orec[..., :3][sel] - pos4[..., :3].astype(np.float64)[sel]
    w /= np.linalg.norm(w, axis=-1, keepdims=True)
    return (w * orec[..., 3:6][sel]).sum(-1)


def compare_trace(occ, orec: np.ndarray, omargin: np.ndarray, valid: np.ndarray, pos4: np.ndarray,
                  what: str = ""):
    r0, r1, tri = gpu_records(occ)
    otri = orec[..., 7].astype(np.int64)
    mism = (tri != otri) & valid
    excused = mism & (omargin < TRACE_MARGIN)
    bad = mism & ~excused
    assert not bad.any(), (
        f"{what}: {bad.sum()} unexplained id mismatches at {np.argwhere(bad)[:8].tolist()}, "
        f"margins {omargin[bad][:8]}")
    assert mism.sum() <= budget(int(valid.sum())), f"{what}: {mism.sum()} grazing mismatches"
    both = valid & (tri >= 0) & (tri == otri)
    if both.any():
        scale = 1.0 + np.abs(orec[..., :3][both]).max(axis=-1)
        t_ref = np.abs(orec[..., 6][both])
        t_err = np.abs(r1[..., 3][both] - orec[..., 6][both])
        # incidence cosine from the oracle record (ray direction = (z - x) / |z - x|)
        graze = DIR_ERR * t_ref / np.maximum(np.abs(_cos_incidence(orec, pos4, both)), 1e-4)
        t_tol = np.maximum(T_RTOL * t_ref, T_ATOL * scale) + graze
        assert np.all(t_err <= t_tol), f"{what}: t err {t_err.max()} (worst ratio {(t_err / t_tol).max()})"
        z_err = np.abs(r0[..., :3][both] - orec[..., :3][both]).max(axis=-1)
        assert np.all(z_err <= POS_ATOL * scale + graze), f"{what}: z err {z_err.max()}"
        n_err = np.abs(r1[..., :3][both] - orec[..., 3:6][both]).max()
        assert n_err <= NRM_ATOL, f"{what}: n_z err {n_err}"
    return {"mismatch": int(mism.sum()), "hits": int(both.sum()),
            "listed": np.argwhere(mism).tolist()}


def compare_out(gpu: np.ndarray, ref: np.ndarray, margin: np.ndarray, valid: np.ndarray,
                what: str = "", atol: float = OUT_ATOL):
    err = np.abs(gpu.astype(np.float64) - ref)
    err[~valid] = 0.0
    over = err > atol
    excused = over & (margin < REUSE_MARGIN)
    bad = over & ~excused
    assert not bad.any(), (
        f"{what}: {bad.sum()} pixels over {atol}: max {err[bad].max():.3g} at "
        f"{np.argwhere(bad)[:6].tolist()} gpu {gpu[bad][:6]} ref {ref[bad][:6]} "
        f"margin {margin[bad][:6]}")
    assert over.sum() <= budget(int(valid.sum())), f"{what}: {over.sum()} marginal pixels"
    # invalid receivers output exactly 1
    assert np.all(gpu[~valid] == 1.0), what
    return {"max_err": float(err.max()), "excused": int(excused.sum())}
