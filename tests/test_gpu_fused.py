"""Fused trace + group reuse (occ_trace_reuse_ao / occ_trace_reuse_shadow): steps 1-3 of
Alg. 1 / Alg. 2 in one kernel for the shared groups 2x1, 2x2, 4x2, 4x4.

Each case is checked three ways on the same seeded inputs:
  - the step-1 records the call also stores, against the oracle's trace (ids equal up to
    the listed grazing flips, t / z / n_z within the FP32 bounds of tests/_parity.py);
  - the estimate against the FP64 oracle's reuse of those records (record-conditioned,
    <= 1e-5 up to listed support-test margins);
  - the estimate against the separate calls (group reuse of the same records), which
    run the same FP32 arithmetic: equal to 1e-6.
Both AO launch paths are covered (one CTA per tile, persistent group refill).
"""
import numpy as np
import pytest

import synth
from tests import _packing as PK
from tests import _parity as P

pytestmark = pytest.mark.gpu

AO, SH = 0, 1
NOREUSE, BIASED, UNBIASED, BOXMEAN = 0, 1, 2, 3
R_C1 = 1.0
LIGHT_C1 = np.array([0.0, 0.5, 3.0, 3.0, 0, 0, 0, -3.0, 0], dtype=np.float32)
GROUPS = [(2, 1), (2, 2), (4, 2), (4, 4)]
AO_PATHS = (1, 2)       # one CTA per 16 x 8 tile, persistent group refill


@pytest.fixture(scope="module")
def occ():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_23122_gb300 import occ as occmod
    return occmod


@pytest.fixture(scope="module")
def ctx(occ):
    return occ.Context(0)


@pytest.fixture(scope="module")
def c1(orc, occ, ctx):
    scene = synth.scene_c1()
    osc = orc.OracleScene(scene.tris)
    pos, nrm, _ = orc.gbuffer(osc, synth.camera_c1().as_array(), 64, 64, scene.eps)
    return {"osc": osc, "bvh": occ.BVH(ctx, scene.tris), "pos": pos, "nrm": nrm,
            "gb": occ.GBuffer.from_numpy(pos, nrm), "R": R_C1, "light": LIGHT_C1}


@pytest.fixture(scope="module")
def terrain_small(orc, occ, ctx):
    scene = synth.scene_terrain(grid=96, n_spheres=20, n_boxes=300, seed=5, sphere_subdiv=2,
                                extent=6.0)
    osc = orc.OracleScene(scene.tris)
    cam = synth.Camera(eye=(0.0, -6.0, 3.0), target=(0.0, 0.0, 0.0), vfov_deg=55.0)
    # 100 x 70: ragged in both directions against the 16 x 8 tiles and every group shape
    pos, nrm, _ = orc.gbuffer(osc, cam.as_array(), 100, 70, scene.eps)
    return {"osc": osc, "bvh": occ.BVH(ctx, scene.tris), "pos": pos, "nrm": nrm,
            "gb": occ.GBuffer.from_numpy(pos, nrm), "R": 0.5, "light": synth.light_c3().as_array()}


def _fused(occ, ctx, s, gb, effect, seed, sample, pat, est, rec=None):
    if effect == AO:
        return occ.occ_trace_reuse_ao(ctx, gb, s["bvh"], s["R"], seed, sample, pat, pat.K, est,
                                      rec=rec)
    return occ.occ_trace_reuse_shadow(ctx, gb, s["bvh"], s["light"], seed, sample, pat, pat.K,
                                      est, rec=rec)


def _separate_reuse(occ, ctx, s, gb, effect, rec, pat, est):
    fn = occ.occ_reuse_ao if effect == AO else occ.occ_reuse_shadow
    return fn(ctx, gb, rec, pat, pat.K, est, bvh=s["bvh"] if est == UNBIASED else None)


def _paths(effect):
    return AO_PATHS if effect == AO else (0,)


@pytest.mark.parametrize("est", [NOREUSE, BIASED, UNBIASED, BOXMEAN])
@pytest.mark.parametrize("effect", [AO, SH])
@pytest.mark.parametrize("which", ["c1", "terrain_small"])
def test_fused_matches_oracle_and_separate_calls(orc, occ, ctx, which, effect, est, request):
    s = request.getfixturevalue(which)
    H, W = s["pos"].shape[:2]
    valid = s["pos"][..., 3] > 0
    seed, sample = 31, 2
    orec, omg = orc.trace(s["osc"], effect, s["pos"], s["nrm"], radius=s["R"], light=s["light"],
                          seed=seed, sample=sample)
    # the separate step 1 on the same rays
    sep_rec = (occ.occ_trace_ao(ctx, s["gb"], s["bvh"], s["R"], seed, sample) if effect == AO else
               occ.occ_trace_shadow(ctx, s["gb"], s["bvh"], s["light"], seed, sample))
    _, _, sep_tri = P.gpu_records(sep_rec)
    try:
        for path in _paths(effect):
            occ.occ_set_tuning(ctx, fused_ao_path=path)
            for gw, gh in GROUPS:
                pat = occ.Pattern.group(gw, gh)
                rec = occ.Occluders.empty(H, W, s["gb"].pos4.device)
                out = _fused(occ, ctx, s, s["gb"], effect, seed, sample, pat, est, rec=rec)
                ctx.sync()
                what = f"{which} effect {effect} est {est} {gw}x{gh} path {path}"
                tr = P.compare_trace(rec, orec, omg, valid, s["pos"], what)
                assert tr["hits"] > 0.03 * valid.sum()
                r0, r1, tri = P.gpu_records(rec)
                # the same closest hits as the separate trace (its own traversal order)
                assert ((tri != sep_tri) & valid).sum() <= P.budget(int(valid.sum())), what
                g = out.cpu().numpy()
                ref, mg = orc.reuse(s["osc"], effect, s["pos"], s["nrm"], P.widen_records(r0, r1),
                                    pat.as_tuple(), est, radius=s["R"], light=s["light"])
                P.compare_out(g, ref, mg, valid, what)
                sep = _separate_reuse(occ, ctx, s, s["gb"], effect, rec, pat, est)
                ctx.sync()
                d = np.abs(g - sep.cpu().numpy())
                assert d.max() <= 1e-6, (what, float(d.max()))
    finally:
        occ.occ_set_tuning(ctx)


@pytest.mark.parametrize("shape", [(1, 1), (7, 3), (33, 17), (16, 8), (61, 37)])
def test_fused_ragged_and_tiny_images(orc, occ, ctx, c1, shape):
    W, H = shape
    x0, y0 = min(10, 64 - W), min(20, 64 - H)
    pos = np.ascontiguousarray(c1["pos"][y0:y0 + H, x0:x0 + W])
    nrm = np.ascontiguousarray(c1["nrm"][y0:y0 + H, x0:x0 + W])
    assert pos.shape[:2] == (H, W)
    gb = occ.GBuffer.from_numpy(pos, nrm)
    valid = pos[..., 3] > 0
    try:
        for effect in (AO, SH):
            for path in _paths(effect):
                occ.occ_set_tuning(ctx, fused_ao_path=path)
                for gw, gh in GROUPS:
                    pat = occ.Pattern.group(gw, gh)
                    for est in (BIASED, UNBIASED):
                        rec = occ.Occluders.empty(H, W, gb.pos4.device)
                        out = _fused(occ, ctx, c1, gb, effect, 8, 1, pat, est, rec=rec)
                        sep = _separate_reuse(occ, ctx, c1, gb, effect, rec, pat, est)
                        ctx.sync()
                        r0, r1, _ = P.gpu_records(rec)
                        ref, mg = orc.reuse(c1["osc"], effect, pos, nrm, P.widen_records(r0, r1),
                                            pat.as_tuple(), est, radius=R_C1, light=LIGHT_C1)
                        what = f"{shape} effect {effect} {gw}x{gh} est {est} path {path}"
                        g = out.cpu().numpy()
                        P.compare_out(g, ref, mg, valid, what)
                        assert np.abs(g - sep.cpu().numpy()).max() <= 1e-6, what
    finally:
        occ.occ_set_tuning(ctx)


def test_fused_without_records_equals_with_records(occ, ctx, terrain_small):
    """Storing the records is a side output: the estimate is the same without it, on both
    AO paths, and with packed records."""
    s = terrain_small
    H, W = s["pos"].shape[:2]
    pat = occ.Pattern.group(4, 2)
    try:
        for effect in (AO, SH):
            for path in _paths(effect):
                occ.occ_set_tuning(ctx, fused_ao_path=path)
                a = _fused(occ, ctx, s, s["gb"], effect, 3, 0, pat, BIASED)
                rec = occ.Occluders.empty(H, W, s["gb"].pos4.device, packed=True)
                b = _fused(occ, ctx, s, s["gb"], effect, 3, 0, pat, BIASED, rec=rec)
                ctx.sync()
                assert occ.torch.equal(a, b), (effect, path)
    finally:
        occ.occ_set_tuning(ctx)


@pytest.mark.parametrize("effect", [AO, SH])
def test_fused_packed_gbuffer(orc, occ, ctx, c1, effect):
    """Packed G-buffer in, packed records out: the estimate matches the oracle on the
    unpacked receivers and the call's own records (unpacked), and the stored records
    match the oracle's trace of the unpacked G-buffer."""
    ppos = PK.pack_gbuffer(c1["pos"], c1["nrm"])
    upos, unrm = PK.unpack_gbuffer(ppos)
    gb = occ.GBuffer(occ.torch.from_numpy(ppos).cuda(), None)
    valid = upos[..., 3] > 0
    try:
        for path in _paths(effect):
            occ.occ_set_tuning(ctx, fused_ao_path=path)
            for gw, gh in GROUPS:
                pat = occ.Pattern.group(gw, gh)
                rec32 = occ.Occluders.empty(64, 64, gb.pos4.device)
                out = _fused(occ, ctx, c1, gb, effect, 17, 0, pat, BIASED, rec=rec32)
                recp = occ.Occluders.empty(64, 64, gb.pos4.device, packed=True)
                out2 = _fused(occ, ctx, c1, gb, effect, 17, 0, pat, BIASED, rec=recp)
                ctx.sync()
                assert occ.torch.equal(out, out2)
                r0, r1, tri = P.gpu_records(rec32)
                orec, omg = orc.trace(c1["osc"], effect, upos, unrm, radius=R_C1, light=LIGHT_C1,
                                      seed=17, sample=0)
                P.compare_trace(rec32, orec, omg, valid, upos, f"packed {gw}x{gh}")
                grec = PK.unpack_records(recp.data[0].cpu().numpy(), upos)
                assert np.array_equal(grec[..., 7], tri.astype(np.float64))
                ref, mg = orc.reuse(c1["osc"], effect, upos, unrm, P.widen_records(r0, r1),
                                    pat.as_tuple(), BIASED, radius=R_C1, light=LIGHT_C1)
                P.compare_out(out.cpu().numpy(), ref, mg, valid, f"packed gbuffer {gw}x{gh}")
    finally:
        occ.occ_set_tuning(ctx)


def test_fused_closed_form_scenes(occ, ctx):
    """No occluder: every estimator gives 1 exactly; a blocker over every receiver gives
    NOREUSE, BIASED (all-blocked guard) and BOXMEAN shadows of exactly 0; all-invalid
    G-buffers give 1 and empty records."""
    pos, nrm = synth.receiver_grid(40, 24, 0.05, z=synth.scene_plane_only().eps)
    gb = occ.GBuffer.from_numpy(pos, nrm)
    light = synth.light_c3().as_array()
    lit = {"bvh": occ.BVH(ctx, synth.scene_plane_only().tris), "R": 1.0, "light": light}
    blk = {"bvh": occ.BVH(ctx, synth.scene_fully_blocked(2.0).tris), "R": 1.0, "light": light}
    try:
        for path in AO_PATHS:
            occ.occ_set_tuning(ctx, fused_ao_path=path)
            for gw, gh in GROUPS:
                pat = occ.Pattern.group(gw, gh)
                for est in (NOREUSE, BIASED, UNBIASED, BOXMEAN):
                    for effect in (AO, SH):
                        out = _fused(occ, ctx, lit, gb, effect, 1, 0, pat, est).cpu().numpy()
                        assert np.all(out == 1.0), (gw, gh, est, effect)
                    if est != UNBIASED:
                        out = _fused(occ, ctx, blk, gb, SH, 1, 0, pat, est).cpu().numpy()
                        assert np.all(out == 0.0), (gw, gh, est)
            empty = occ.GBuffer.from_numpy(np.zeros((20, 30, 4), np.float32),
                                           np.zeros((20, 30, 4), np.float32))
            rec = occ.Occluders.empty(20, 30, empty.pos4.device)
            out = _fused(occ, ctx, blk, empty, AO, 1, 0, occ.Pattern.group(4, 2), BIASED, rec=rec)
            ctx.sync()
            assert np.all(out.cpu().numpy() == 1.0)
            assert np.all(rec.tri.cpu().numpy() == -1)
    finally:
        occ.occ_set_tuning(ctx)


def test_fused_arguments(occ, ctx, c1):
    gb, bvh = c1["gb"], c1["bvh"]
    with pytest.raises(occ.OccError, match="UNSUPPORTED"):
        occ.occ_trace_reuse_ao(ctx, gb, bvh, 1.0, 1, 0, occ.Pattern.group(3, 2), 6, BIASED)
    with pytest.raises(occ.OccError, match="UNSUPPORTED"):
        occ.occ_trace_reuse_ao(ctx, gb, bvh, 1.0, 1, 0, occ.Pattern.box(3, 3), 9, BIASED)
    with pytest.raises(occ.OccError, match="UNSUPPORTED"):
        occ.occ_trace_reuse_shadow(ctx, gb, bvh, LIGHT_C1, 1, 0,
                                   occ.Pattern.offsets_of(synth.disk_offsets(8, 15.0, seed=3)),
                                   8, BIASED)
    with pytest.raises(occ.OccError, match="INVALID_ARG"):
        occ.occ_trace_reuse_ao(ctx, gb, bvh, 1.0, 1, 0, occ.Pattern.group(4, 2), 7, BIASED)
    with pytest.raises(occ.OccError, match="INVALID_ARG"):
        occ.occ_trace_reuse_shadow(ctx, gb, bvh, LIGHT_C1, 1, 0, occ.Pattern.group(4, 2), 8, 4)
    with pytest.raises(occ.OccError, match="INVALID_ARG"):
        occ.occ_trace_reuse_ao(ctx, gb, bvh, -1.0, 1, 0, occ.Pattern.group(4, 2), 8, BIASED)
    with pytest.raises(occ.OccError, match="INVALID_ARG"):
        occ.occ_set_tuning(ctx, fused_ao_path=3)
    ctx.sync()
