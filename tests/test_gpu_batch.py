"""Batched frames (occ_frame_batch), captured batches (occ_batch_*), runtime tuning and
the autotuner.

A batch of uneven views (sizes, effects, estimators, patterns, formats) must give, view by
view, the records of the per-view trace calls bit for bit and the estimate of the
per-view reuse calls (bit for bit where both run the per-receiver kernel; within FP32
summation-order rounding where the per-view call ran the warp-cooperative group kernel);
and, on its own records, the oracle's estimate within the parity tolerance.
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
    return {"osc": osc, "bvh": occ.BVH(ctx, scene.tris), "pos": pos, "nrm": nrm}


def _pattern(occ, name):
    return {
        "group2x2": lambda: occ.Pattern.group(2, 2), "group4x2": lambda: occ.Pattern.group(4, 2),
        "group4x4": lambda: occ.Pattern.group(4, 4), "group3x2": lambda: occ.Pattern.group(3, 2),
        "box3x3": lambda: occ.Pattern.box(3, 3),
        "disk8": lambda: occ.Pattern.offsets_of(synth.disk_offsets(8, 15.0, seed=3)),
        "disk16": lambda: occ.Pattern.offsets_of(synth.disk_offsets(16, 6.0, seed=4)),
    }[name]()


# (x0, y0, W, H) crop of the 64x64 C1 G-buffer, effect, estimator, pattern, packed formats
SPECS = [
    ((0, 0, 64, 64), AO, BIASED, "group4x2", False),
    ((10, 20, 33, 17), SH, UNBIASED, "box3x3", False),
    ((5, 30, 7, 3), AO, NOREUSE, "disk8", False),
    ((0, 0, 64, 64), SH, BIASED, "disk16", True),
    ((12, 8, 40, 24), AO, BOXMEAN, "group3x2", False),
    ((30, 30, 1, 1), SH, BIASED, "group2x2", False),
    ((0, 0, 64, 64), AO, UNBIASED, "group4x4", False),
    ((3, 1, 50, 61), SH, BIASED, "box3x3", True),
]


def _make_views(occ, c1, specs=SPECS, seed0=100):
    import torch
    views, host = [], []
    for i, ((x0, y0, W, H), eff, est, pname, packed) in enumerate(specs):
        pos = np.ascontiguousarray(c1["pos"][y0:y0 + H, x0:x0 + W])
        nrm = np.ascontiguousarray(c1["nrm"][y0:y0 + H, x0:x0 + W])
        if packed:
            ppos = PK.pack_gbuffer(pos, nrm)
            gb = occ.GBuffer(torch.from_numpy(ppos).cuda(), None)
            pos, nrm = PK.unpack_gbuffer(ppos)        # what the kernels see
        else:
            gb = occ.GBuffer.from_numpy(pos, nrm)
        pat = _pattern(occ, pname)
        views.append(occ.View(gb=gb, rec=occ.Occluders.empty(H, W, packed=packed),
                              out=torch.full((H, W), -7.0, device="cuda"), effect=eff,
                              radius=R_C1, light=LIGHT_C1 if eff == SH else None,
                              seed=seed0 + i, sample=i, pattern=pat, estimator=est))
        host.append({"pos": pos, "nrm": nrm, "packed": packed, "pname": pname})
    return views, host


def _per_view(occ, ctx, c1, v):
    """The same view through the per-view C-ABI calls."""
    if v.effect == AO:
        o = occ.occ_trace_ao(ctx, v.gb, c1["bvh"], v.radius, v.seed, v.sample, packed=v.rec.packed)
    else:
        o = occ.occ_trace_shadow(ctx, v.gb, c1["bvh"], v.light, v.seed, v.sample,
                                 packed=v.rec.packed)
    fn = occ.occ_reuse_ao if v.effect == AO else occ.occ_reuse_shadow
    out = fn(ctx, v.gb, o, v.pattern, v.pattern.K, v.estimator,
             bvh=c1["bvh"] if v.estimator == UNBIASED else None)
    return o, out


def _bits(rec):
    """Record planes as raw words (a miss stores tri = -1, a NaN pattern, in a float slot)."""
    return rec.data.cpu().numpy().view(np.uint32)


def _oracle_records(v, h):
    d = v.rec.data.cpu().numpy()
    if h["packed"]:
        return PK.unpack_records(d[0], h["pos"])
    return P.widen_records(d[0], d[1])


def _uses_group_kernel(v, occ):
    """Whether the per-view reuse call ran the warp-cooperative group kernel."""
    p = v.pattern
    return (p.kind == occ.OCC_PAT_GROUP and (p.gw, p.gh) in ((2, 1), (2, 2), (4, 2), (4, 4))
            and v.gb.packed == v.rec.packed and v.estimator in (BIASED, UNBIASED))


def test_batch_equals_per_view_calls_and_oracle(orc, occ, ctx, c1):
    views, host = _make_views(occ, c1)
    occ.occ_set_tuning(ctx, reuse_window_path=2)     # per-view windows on the per-receiver kernel
    try:
        occ.occ_frame_batch(ctx, c1["bvh"], views)
        refs = [_per_view(occ, ctx, c1, v) for v in views]
        ctx.sync()
    finally:
        occ.occ_set_tuning(ctx)
    for i, (v, h, (o, out)) in enumerate(zip(views, host, refs)):
        assert v.rec.meta.seed == v.seed and v.rec.meta.sample == v.sample
        assert np.array_equal(_bits(v.rec), _bits(o)), f"view {i} records"
        got, want = v.out.cpu().numpy(), out.cpu().numpy()
        if _uses_group_kernel(v, occ):
            assert np.abs(got - want).max() <= 2e-6, (i, np.abs(got - want).max())
        else:
            assert np.array_equal(got, want), (i, np.abs(got - want).max())
        # the batch's estimate against the oracle on the batch's own records
        valid = h["pos"][..., 3] > 0
        ref, mg = orc.reuse(c1["osc"], v.effect, h["pos"], h["nrm"], _oracle_records(v, h),
                            v.pattern.as_tuple(), v.estimator, radius=R_C1, light=LIGHT_C1)
        P.compare_out(got, ref, mg, valid, f"batch view {i} ({h['pname']})")


def test_batch_results_do_not_depend_on_the_mix(occ, ctx, c1):
    """A view alone and the same view inside a batch give the same bits."""
    views, _ = _make_views(occ, c1)
    occ.occ_frame_batch(ctx, c1["bvh"], views)
    for i in (1, 3, 5):
        alone, _ = _make_views(occ, c1, [SPECS[i]], seed0=100 + i)
        alone[0].sample = views[i].sample
        occ.occ_frame_batch(ctx, c1["bvh"], alone)
        ctx.sync()
        assert np.array_equal(alone[0].out.cpu().numpy(), views[i].out.cpu().numpy())
        assert np.array_equal(_bits(alone[0].rec), _bits(views[i].rec))


@pytest.mark.parametrize("per_sm", [1, 3, 16])
def test_batch_ctas_per_sm_does_not_change_results(occ, ctx, c1, per_sm):
    views, _ = _make_views(occ, c1)
    occ.occ_frame_batch(ctx, c1["bvh"], views)
    ctx.sync()
    want = [v.out.clone() for v in views]
    occ.occ_set_tuning(ctx, batch_ctas_per_sm=per_sm)
    try:
        for v in views:
            v.out.fill_(-1.0)
        occ.occ_frame_batch(ctx, c1["bvh"], views)
        ctx.sync()
    finally:
        occ.occ_set_tuning(ctx)
    for v, w in zip(views, want):
        assert np.array_equal(v.out.cpu().numpy(), w.cpu().numpy())


def test_graph_replay_equals_direct_batch(occ, ctx, c1):
    views, _ = _make_views(occ, c1)
    batch = occ.Batch(ctx, c1["bvh"], views)
    n = len(views)
    results = {}
    for trial, (s0, m0) in enumerate(((7, 0), (9, 5), (7, 0))):
        seeds = np.arange(n, dtype=np.uint64) + np.uint64(s0)
        samples = np.arange(n, dtype=np.uint32) + np.uint32(m0)
        batch.replay(seeds, samples)
        ctx.sync()
        got = [v.out.cpu().numpy().copy() for v in views]
        recs = [_bits(v.rec) for v in views]
        direct, _ = _make_views(occ, c1)
        for v, s, m in zip(direct, seeds, samples):
            v.seed, v.sample = int(s), int(m)
        occ.occ_frame_batch(ctx, c1["bvh"], direct)
        ctx.sync()
        for i, v in enumerate(direct):
            assert np.array_equal(got[i], v.out.cpu().numpy()), (trial, i)
            assert np.array_equal(recs[i], _bits(v.rec)), (trial, i)
        results[trial] = got
    # new seeds change the estimate; the old ones give it back
    assert any(not np.array_equal(a, b) for a, b in zip(results[0], results[1]))
    assert all(np.array_equal(a, b) for a, b in zip(results[0], results[2]))
    batch.free()


def test_batch_arguments_rejected(occ, ctx, c1):
    views, _ = _make_views(occ, c1, SPECS[:2])
    with pytest.raises(occ.OccError, match="INVALID_ARG"):
        occ.occ_frame_batch(ctx, c1["bvh"], [])
    big, _ = _make_views(occ, c1, [((0, 0, 64, 64), AO, BIASED, "group4x2", False)])
    big[0].pattern = occ.Pattern.box(5, 5)                       # K = 25 > 16
    with pytest.raises(occ.OccError, match="UNSUPPORTED"):
        occ.occ_frame_batch(ctx, c1["bvh"], big)
    bad, _ = _make_views(occ, c1, SPECS[:1])
    bad[0].rec = occ.Occluders.empty(63, 64)                     # records of another size
    with pytest.raises(occ.OccError, match="INVALID_ARG"):
        occ.occ_frame_batch(ctx, c1["bvh"], bad)
    with pytest.raises(occ.OccError, match="INVALID_ARG"):
        occ.occ_set_tuning(ctx, reuse_tile_rows=5)
    with pytest.raises(occ.OccError, match="INVALID_ARG"):
        occ.occ_set_tuning(ctx, batch_ctas_per_sm=17)
    occ.occ_frame_batch(ctx, c1["bvh"], views)                   # the context still works
    ctx.sync()


# --------------------------------------------------------------------------------------
# Runtime tuning of the window path: every choice stays at parity with the oracle
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("cfg", [dict(reuse_window_path=1, reuse_tile_rows=4),
                                 dict(reuse_window_path=1, reuse_tile_rows=8),
                                 dict(reuse_window_path=1, reuse_tile_rows=16),
                                 dict(reuse_window_path=3, reuse_tile_rows=4),
                                 dict(reuse_window_path=3, reuse_tile_rows=8),
                                 dict(reuse_window_path=3, reuse_tile_rows=16),
                                 dict(reuse_window_path=2)])
@pytest.mark.parametrize("pname", ["box3x3", "disk8"])
@pytest.mark.parametrize("effect", [AO, SH])
def test_tuning_choices_match_oracle(orc, occ, ctx, c1, cfg, pname, effect):
    pat = _pattern(occ, pname)
    orec, _ = orc.trace(c1["osc"], effect, c1["pos"], c1["nrm"], radius=R_C1, light=LIGHT_C1,
                        seed=61, sample=1)
    r0, r1 = P.to_f32_records(orec)
    o = occ.Occluders.from_numpy(r0, r1, effect, radius=R_C1, light=LIGHT_C1)
    gb = occ.GBuffer.from_numpy(c1["pos"], c1["nrm"])
    fn = occ.occ_reuse_ao if effect == AO else occ.occ_reuse_shadow
    occ.occ_set_tuning(ctx, **cfg)
    try:
        assert {k: occ.occ_get_tuning(ctx)[k] for k in cfg} == cfg
        g = fn(ctx, gb, o, pat, pat.K, BIASED)
        ctx.sync()
    finally:
        occ.occ_set_tuning(ctx)
    ref, mg = orc.reuse(c1["osc"], effect, c1["pos"], c1["nrm"], P.widen_records(r0, r1),
                        pat.as_tuple(), BIASED, radius=R_C1, light=LIGHT_C1)
    P.compare_out(g.cpu().numpy(), ref, mg, c1["pos"][..., 3] > 0, f"tuning {cfg} {pname}")


@pytest.mark.parametrize("cfg", [dict(trace_path=1), dict(trace_path=2),
                                 dict(trace_path=2, trace_refill=1, trace_ctas_per_sm=1),
                                 dict(trace_path=2, trace_refill=32, trace_ctas_per_sm=3),
                                 dict(trace_path=2, trace_order=2),
                                 dict(trace_path=2, trace_order=2, trace_refill=8),
                                 dict(group_prefetch=1), dict(group_prefetch=3)])
@pytest.mark.parametrize("effect", [AO, SH])
def test_trace_and_group_tuning_choices_are_bit_identical(occ, ctx, c1, cfg, effect):
    """Every trace launch choice (kernel, refill threshold, CTAs per SM) writes the same
    records, and every group prefetch choice the same estimate, as the defaults."""
    gb = occ.GBuffer.from_numpy(c1["pos"], c1["nrm"])

    def run():
        o = (occ.occ_trace_ao(ctx, gb, c1["bvh"], R_C1, 13, 2) if effect == AO else
             occ.occ_trace_shadow(ctx, gb, c1["bvh"], LIGHT_C1, 13, 2))
        fn = occ.occ_reuse_ao if effect == AO else occ.occ_reuse_shadow
        g = fn(ctx, gb, o, occ.Pattern.group(4, 2), 8, BIASED)
        ctx.sync()
        return o.data.clone(), g
    rec0, out0 = run()
    occ.occ_set_tuning(ctx, **cfg)
    try:
        assert {k: occ.occ_get_tuning(ctx)[k] for k in cfg} == cfg
        rec1, out1 = run()
    finally:
        occ.occ_set_tuning(ctx)
    # records compared as bits (a miss's triangle id -1 is a NaN pattern as a float)
    i32 = occ.torch.int32
    assert occ.torch.equal(rec0.view(i32), rec1.view(i32)) and occ.torch.equal(out0, out1)


def test_batch_of_tiled_views_matches_row_major(occ, ctx, c1):
    """Every view of a batch given as a tiled G-buffer (occ_tile_gbuffer) gives the same
    records and estimates, bit for bit, as the same batch with row-major G-buffers (views of
    every size, both formats, every estimator)."""
    views, _ = _make_views(occ, c1)
    tviews, _ = _make_views(occ, c1)
    for v in tviews:
        v.gb = occ.occ_tile_gbuffer(ctx, v.gb)
    occ.occ_frame_batch(ctx, c1["bvh"], views)
    occ.occ_frame_batch(ctx, c1["bvh"], tviews)
    ctx.sync()
    for i, (a, b) in enumerate(zip(views, tviews)):
        assert b.gb.tiled
        assert np.array_equal(_bits(a.rec), _bits(b.rec)), f"view {i} records"
        assert np.array_equal(a.out.cpu().numpy(), b.out.cpu().numpy()), f"view {i} estimate"


def test_autotuner_picks_caches_and_reapplies(occ, ctx, c1, tmp_path, monkeypatch):
    from paper_2607_23122_gb300 import autotune
    monkeypatch.setenv("OCC_TUNE_CACHE", str(tmp_path / "tune.json"))
    gb = occ.GBuffer.from_numpy(c1["pos"], c1["nrm"])
    o = occ.occ_trace_ao(ctx, gb, c1["bvh"], R_C1, 3, 0)
    pat = _pattern(occ, "disk8")
    out = occ.torch.empty((64, 64), device="cuda")
    entry = autotune.tune_reuse(ctx, gb, o, pat, BIASED, out, iters=3)
    assert entry["best"] in autotune.REUSE_CANDIDATES
    assert len(entry["timings"]) == len(autotune.REUSE_CANDIDATES)
    assert all(t["ms"] > 0 for t in entry["timings"])
    tuned = occ.occ_get_tuning(ctx)
    assert all(tuned[k] == v for k, v in entry["best"].items())
    # a second call reads the cache and measures nothing
    occ.occ_set_tuning(ctx)
    timer = autotune._time
    monkeypatch.setattr(autotune, "_time", lambda *a, **k: pytest.fail("re-measured"))
    again = autotune.tune_reuse(ctx, gb, o, pat, BIASED, out)
    assert again["best"] == entry["best"]
    assert occ.occ_get_tuning(ctx) == tuned
    monkeypatch.setattr(autotune, "_time", timer)
    views, _ = _make_views(occ, c1, SPECS[:3])
    b = autotune.tune_batch(ctx, c1["bvh"], views, iters=2, use_cache=False)
    assert b["best"] in autotune.BATCH_CANDIDATES
    occ.occ_set_tuning(ctx)
    rec = occ.Occluders.empty(64, 64)
    t = autotune.tune_trace(ctx, gb, c1["bvh"], AO, rec, radius=R_C1, iters=2)
    assert len(t["timings"]) == len(autotune.TRACE_CANDIDATES)
    assert all(occ.occ_get_tuning(ctx)[k] == v for k, v in t["best"].items())
    key = autotune.trace_key(gb, rec, c1["bvh"], AO)
    assert autotune.load_cache()[key]["best"] == t["best"]
    occ.occ_set_tuning(ctx)
    g = autotune.tune_reuse(ctx, gb, o, occ.Pattern.group(4, 2), BIASED, out, iters=2,
                            use_cache=False)
    assert g["best"] in autotune.GROUP_CANDIDATES
    occ.occ_set_tuning(ctx)
    # G-buffer layout: row-major or a tiled copy, timed over a frame; the cached choice comes
    # back with the G-buffer to use
    lay = autotune.tune_layout(ctx, gb, c1["bvh"], AO, occ.Pattern.group(4, 2), BIASED, rec, out,
                               radius=R_C1, iters=2)
    assert [t["config"]["gbuffer_layout"] for t in lay["timings"]] == list(autotune.LAYOUT_CANDIDATES)
    assert lay["gbuffer"].tiled == (lay["best"]["gbuffer_layout"] == "tiled")
    monkeypatch.setattr(autotune, "_time", lambda *a, **k: pytest.fail("re-measured"))
    lay2 = autotune.tune_layout(ctx, gb, c1["bvh"], AO, occ.Pattern.group(4, 2), BIASED, rec, out,
                                radius=R_C1)
    assert lay2["best"] == lay["best"] and lay2["gbuffer"].tiled == lay["gbuffer"].tiled
    monkeypatch.setattr(autotune, "_time", timer)
    ctx.sync()
