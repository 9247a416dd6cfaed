"""RelMSE as the quality harness computes it (no GPU)."""
import numpy as np


def test_relmse_definition():
    from paper_2607_23122_gb300 import quality as Q
    ref = np.array([[0.5, 0.0], [1.0, 0.2]])
    est = np.array([[0.4, 0.1], [1.0, 0.2]])
    valid = np.array([[True, True], [True, False]])
    want = np.mean([0.01 / (0.25 + 1e-3), 0.01 / (0.0 + 1e-3), 0.0])
    assert abs(Q.relmse(est, ref, valid) - want) < 1e-12


def test_region_errors_split_the_image():
    from paper_2607_23122_gb300 import quality as Q
    ref = np.array([[0.0, 0.5], [1.0, 0.25]])
    est = np.array([[0.1, 0.5], [0.9, 0.5]])
    valid = np.ones((2, 2), dtype=bool)
    b = Q.region_errors(est, ref, valid)
    assert (b["umbra"]["pixels"], b["penumbra"]["pixels"], b["lit"]["pixels"]) == (1, 2, 1)
    assert abs(b["umbra"]["mse"] - 0.01) < 1e-15 and abs(b["lit"]["bias"] + 0.1) < 1e-12
    assert abs(b["penumbra"]["mse"] - 0.0625 / 2) < 1e-15
    assert abs(sum(v["relmse_share"] for v in b.values()) - 1.0) < 1e-12


def test_biased_shadow_reuse_by_region_on_the_half_plane(orc):
    """Sec. 6.2 shadows, where the estimators differ: on the half-plane blocker (closed-form
    reference clamp((X* - a) / w, 0, 1)), per-sample errors of the oracle's estimators by
    region.  Biased Occ(8) on 4x2 groups is exactly 0 in the umbra (the all-blocked guard of
    Sec. 4.4) and several times below no reuse in the penumbra; the unbiased estimator has no
    guard and carries umbra variance around 0.  So a RelMSE that divides umbra errors by
    eps = 1e-3 rewards no reuse (exactly 0 there) wherever a group straddles a shadow edge,
    which fragmented shadows of many small occluders make common."""
    import math

    import synth
    hb = 2.0
    scene = synth.scene_half_plane(hb)
    sc = orc.OracleScene(scene.tris)
    light = np.array([0.5, 0.0, 4.0, 1.0, 0, 0, 0, -0.5, 0], dtype=np.float32)
    pos, nrm = synth.receiver_grid(96, 8, 0.021, z=scene.eps, origin=(-0.5, 0.0))
    x = pos[..., 0].astype(np.float64)
    zr = float(pos[0, 0, 2])
    lam = (hb - zr) / (4.0 - zr)
    ref = np.clip(-x * (1 - lam) / lam, 0.0, 1.0)
    umbra, pen = ref == 0.0, (ref > 0) & (ref < 1)
    assert umbra.sum() > 100 and pen.sum() > 200
    M = 128
    err = {}
    for name, pat, est in (("noreuse", (0, 1, 1, None), 0), ("biased", (0, 4, 2, None), 1),
                           ("unbiased", (0, 4, 2, None), 2)):
        mean, var = orc.accumulate(sc, 1, pos, nrm, pat, est, light=light, seed=21, sample0=0, M=M)
        mse = var * (M - 1) / M + (mean - ref) ** 2
        err[name] = {"umbra": mse[umbra].mean(), "penumbra": mse[pen].mean(),
                     "bias": abs((mean - ref)[pen].mean()), "sig": math.sqrt(var[pen].mean() / M)}
    assert err["noreuse"]["umbra"] == 0.0 and err["biased"]["umbra"] == 0.0
    assert err["unbiased"]["umbra"] > 1e-3
    assert err["biased"]["penumbra"] < 0.3 * err["noreuse"]["penumbra"]
    assert err["biased"]["bias"] < 5 * err["biased"]["sig"]
