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

End to end (each side reuses its own trace's records) the FP32 rounding of the records
propagates into the estimate: z is good to a few FP32 ulps of |z| (the watertight test
works on vertices relative to the ray origin), and the densities go as 1/r^4 in the pair
distance r.  compare_end_to_end therefore lists every pixel over OUT_ATOL with its minimum
pair distance, its oracle margin and its conditioning kappa: the largest change of the FP64
estimate when every record's z moves by PERTURB_ULPS FP32 ulps in a seeded random
direction (computed by the oracle alone, from its own records).  A listed pixel is
explained when kappa >= OUT_ATOL / 4 (ill-conditioned at FP32 precision) or its margin is
below FLIP_MARGIN (a support test within FP32 reach of its threshold); unexplained pixels
may not exceed DISAGREE_FRAC of the pixels considered, and neither may all listed pixels
where the scene's conditioning allows it (the small scene).  Pixels whose neighbour set
holds a listed trace disagreement are excluded and counted.
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
PERTURB_ULPS = 2.0
FLIP_MARGIN = 2e-3


def ulp32(x: np.ndarray) -> np.ndarray:
    """FP32 unit in the last place of |x| (normal range)."""
    x = np.maximum(np.abs(np.asarray(x, dtype=np.float64)), np.finfo(np.float32).tiny)
    return np.exp2(np.floor(np.log2(x)) - 23)


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
    n_graze = 0
    z_ulps = 0.0
    if both.any():
        scale = 1.0 + np.abs(orec[..., :3][both]).max(axis=-1)
        t_ref = np.abs(orec[..., 6][both])
        t_err = np.abs(r1[..., 3][both] - orec[..., 6][both])
        # incidence cosine from the oracle record (ray direction = (z - x) / |z - x|)
        graze = DIR_ERR * t_ref / np.maximum(np.abs(_cos_incidence(orec, pos4, both)), 1e-4)
        base = np.maximum(T_RTOL * t_ref, T_ATOL * scale)
        t_tol = base + graze
        assert np.all(t_err <= t_tol), f"{what}: t err {t_err.max()} (worst ratio {(t_err / t_tol).max()})"
        z_err = np.abs(r0[..., :3][both] - orec[..., :3][both]).max(axis=-1)
        assert np.all(z_err <= POS_ATOL * scale + graze), f"{what}: z err {z_err.max()}"
        # hits whose distance needs the grazing term: FP32 direction error turned into a
        # distance error by incidence angles near 90 degrees; they must stay rare
        need = (t_err > base) | (z_err > POS_ATOL * scale)
        n_graze = int(need.sum())
        assert n_graze <= budget(int(both.sum())), f"{what}: {n_graze} hits need the grazing term"
        z_ulps = float(np.quantile(z_err / ulp32(np.abs(orec[..., :3][both]).max(axis=-1)), 0.999))
        n_err = np.abs(r1[..., :3][both] - orec[..., 3:6][both]).max()
        assert n_err <= NRM_ATOL, f"{what}: n_z err {n_err}"
    return {"mismatch": int(mism.sum()), "hits": int(both.sum()), "grazing": n_graze,
            "z_err_ulps_p999": z_ulps, "listed": np.argwhere(mism).tolist(), "flip_mask": mism}


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


# --------------------------------------------------------------------------------------
# End to end (P5): each side reuses the records of its own trace
# --------------------------------------------------------------------------------------

def member_offsets(pattern, W: int, H: int):
    """Per member slot of every receiver: (x, y, inside) arrays [H, W] (N_i of Eq. 8 before
    dropping invalid members), pattern = (kind, gw, gh, offsets) as the oracle takes it."""
    kind, gw, gh, off = pattern
    ys, xs = np.mgrid[0:H, 0:W]
    if kind == 0:
        bx, by = (xs // gw) * gw, (ys // gh) * gh
        slots = [(bx + i % gw, by + i // gw) for i in range(gw * gh)]
    elif kind == 1:
        slots = [(xs + dx, ys + dy) for dy in range(-((gh - 1) // 2), gh // 2 + 1)
                 for dx in range(-((gw - 1) // 2), gw // 2 + 1)]
    else:
        slots = [(xs, ys)] + [(xs + int(a), ys + int(b)) for a, b in np.asarray(off).reshape(-1, 2)]
    out = []
    for mx, my in slots:
        ok = (mx >= 0) & (mx < W) & (my >= 0) & (my < H)
        out.append((np.clip(mx, 0, W - 1), np.clip(my, 0, H - 1), ok))
    return out


def neighbourhood_stats(pos4: np.ndarray, orec: np.ndarray, pattern, flips: np.ndarray):
    """(r_min [H, W], flip_nb [H, W]): the smallest distance between a member's receiver and a
    member's occluder point, and whether N_i holds a pixel with a trace disagreement."""
    H, W = pos4.shape[:2]
    valid = pos4[..., 3] > 0
    mem = [(mx, my, ok & valid[my, mx]) for mx, my, ok in member_offsets(pattern, W, H)]
    rmin = np.full((H, W), np.inf)
    flip_nb = np.zeros((H, W), dtype=bool)
    xk = [pos4[my, mx, :3].astype(np.float64) for mx, my, _ in mem]
    for jx, jy, jok in mem:
        flip_nb |= jok & flips[jy, jx]
        hit = jok & (orec[jy, jx, 7] >= 0)
        z = orec[jy, jx, :3]
        for (_, _, kok), x in zip(mem, xk):
            d = np.sqrt(((z - x) ** 2).sum(-1))
            rmin = np.where(hit & kok, np.minimum(rmin, d), rmin)
    return rmin, flip_nb


def conditioning(orc, scene, effect, pos4, nrm4, orec, pattern, est, radius=0.0, light=None,
                 n_draws: int = 2, seed: int = 12345):
    """kappa [H, W]: the largest change of the oracle's estimate over n_draws seeded random
    moves of every hit record's z by PERTURB_ULPS FP32 ulps of its largest coordinate per axis
    (signs random).  Computed from the oracle's own records only."""
    base, _ = orc.reuse(scene, effect, pos4, nrm4, orec, pattern, est, radius=radius, light=light)
    rng = np.random.default_rng(seed)
    hit = orec[..., 7] >= 0
    step = PERTURB_ULPS * ulp32(np.abs(orec[..., :3]).max(axis=-1))
    kappa = np.zeros(base.shape)
    for _ in range(n_draws):
        rec = orec.copy()
        sgn = rng.choice([-1.0, 1.0], size=orec[..., :3].shape)
        rec[..., :3] += np.where(hit[..., None], sgn * step[..., None], 0.0)
        o, _ = orc.reuse(scene, effect, pos4, nrm4, rec, pattern, est, radius=radius, light=light)
        kappa = np.maximum(kappa, np.abs(o - base))
    return kappa


def compare_end_to_end(gpu: np.ndarray, ref: np.ndarray, on_gpu_rec: np.ndarray,
                       margin: np.ndarray, kappa: np.ndarray, rmin: np.ndarray,
                       flip_nb: np.ndarray, valid: np.ndarray, what: str = "",
                       strict_count: bool = False) -> dict:
    """P5 on the pixels whose neighbour set holds no trace disagreement (see the module
    docstring).  ref: oracle estimate on the oracle's records; on_gpu_rec: oracle estimate on
    the GPU's records (the GPU's reuse must match it to OUT_ATOL: P4 on its own records)."""
    gpu = gpu.astype(np.float64)
    cons = valid & ~flip_nb
    err = np.where(cons, np.abs(gpu - ref), 0.0)
    p4 = np.where(cons, np.abs(gpu - on_gpu_rec), 0.0)
    p4_bad = (p4 > OUT_ATOL) & (margin >= REUSE_MARGIN)
    assert p4_bad.sum() <= budget(int(cons.sum())), (
        f"{what}: GPU reuse vs oracle on the GPU's records: {p4_bad.sum()} pixels over "
        f"{OUT_ATOL}, max {p4.max():.3g}")
    listed = cons & (err > OUT_ATOL)
    explained = listed & ((kappa >= OUT_ATOL / 4) | (margin < FLIP_MARGIN))
    unexplained = listed & ~explained
    n_cons = int(cons.sum())
    res = {"pixels": int(valid.sum()), "excluded_flip_nb": int((valid & flip_nb).sum()),
           "considered": n_cons, "max_err": float(err.max()) if n_cons else 0.0,
           "p9999": float(np.quantile(err[cons], 0.9999)) if n_cons else 0.0,
           "over": int(listed.sum()), "over_frac": float(listed.sum() / max(1, n_cons)),
           "unexplained": int(unexplained.sum()), "p4_max": float(p4.max()) if n_cons else 0.0,
           "listed": [(int(y), int(x), float(err[y, x]), float(rmin[y, x]), float(margin[y, x]),
                       float(kappa[y, x])) for y, x in np.argwhere(listed)]}
    if listed.any():
        res["rmin_listed_q50_q90"] = [float(v) for v in np.quantile(rmin[listed], [0.5, 0.9])]
        res["rmin_all_q50"] = float(np.median(rmin[cons & np.isfinite(rmin)]))
    assert res["unexplained"] <= budget(n_cons), (
        f"{what}: {res['unexplained']} pixels over {OUT_ATOL} neither ill-conditioned nor at a "
        f"support margin: {[l for l in res['listed'] if l[5] < OUT_ATOL / 4 and l[4] >= FLIP_MARGIN][:6]}")
    if strict_count:
        assert res["over"] <= budget(n_cons), f"{what}: {res['over']} pixels over {OUT_ATOL}"
    return res
