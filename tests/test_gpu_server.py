"""Serving loop (occ_server_*) on the GPU: each result is the same alone and in a mix of
requests admitted while others run; results equal the direct trace + reuse calls; the
budget bounds admitted bytes; deadlines, cancellation and argument checks."""
import threading
import time

import numpy as np
import pytest

import synth
from tests import _parity as P

pytestmark = pytest.mark.gpu

AO, SH = 0, 1
NOREUSE, BIASED, UNBIASED, BOXMEAN = 0, 1, 2, 3
OK, INVALID, OOM, TIMEOUT, CANCELLED = 0, 1, 3, 4, 8
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
    return {"scene": scene, "osc": osc, "bvh": occ.BVH(ctx, scene.tris), "pos": pos, "nrm": nrm}


def _pattern(occ, K):
    return {4: occ.Pattern.group(2, 2), 8: occ.Pattern.offsets_of(synth.disk_offsets(8, 15.0, 3)),
            9: occ.Pattern.box(3, 3), 16: occ.Pattern.group(4, 4),
            17: occ.Pattern.offsets_of(synth.disk_offsets(17, 9.0, 6))}[K]


def _cams():
    base = synth.camera_c1()
    return [base, synth.Camera(eye=(4.0, -4.0, 3.0), target=(0.0, 0.0, 0.2), vfov_deg=60.0),
            synth.Camera(eye=(-5.0, 1.0, 2.5), target=(0.5, 0.0, 0.4), vfov_deg=45.0)]


# W, H, effect, K, estimator, packed, camera index, device output
MIX = [
    (64, 64, AO, 8, BIASED, 0, 0, False),
    (33, 17, SH, 9, UNBIASED, 0, 1, True),
    (128, 96, AO, 16, BIASED, 1, 2, False),
    (16, 8, SH, 4, BIASED, 1, 0, False),
    (100, 37, AO, 4, UNBIASED, 0, 1, True),
    (96, 80, SH, 8, BIASED, 0, 2, False),
    (1, 1, AO, 9, BOXMEAN, 0, 0, False),
    (72, 40, SH, 16, NOREUSE, 1, 1, True),
    (80, 60, AO, 17, BIASED, 0, 2, False),      # K > 16: per-view kernels at any size
    (48, 48, SH, 9, BIASED, 1, 0, False),
]


def _submit(occ, srv, c1, spec, seed, sample=0, deadline_ns=0):
    import torch
    W, H, eff, K, est, packed, cam, dev = spec
    out = (torch.full((H, W), float("nan"), device="cuda") if dev
           else torch.full((H, W), float("nan")).pin_memory())
    rid = srv.submit(W, H, eff, _pattern(occ, K), est, out, radius=1.0,
                     light=LIGHT_C1 if eff == SH else None, seed=seed, sample=sample,
                     packed=bool(packed), camera=_cams()[cam].as_array(), eps=c1["scene"].eps,
                     deadline_ns=deadline_ns)
    return rid, out


def test_each_result_is_the_same_alone_and_in_the_mix(occ, ctx, c1):
    srv = occ.Server(ctx, c1["bvh"], max_views_per_batch=3, max_inflight=2, batch_max_px=5000,
                     batch_window_us=20000)
    try:
        alone = {}
        for i, spec in enumerate(MIX):
            rid, out = _submit(occ, srv, c1, spec, seed=500 + i, sample=i)
            res = srv.wait([rid])[rid]
            assert res["status"] == OK, res
            alone[i] = out.cpu().numpy().copy()
            # every pixel written; the estimator is not clamped, so only 1 bounds it
            assert np.all(np.isfinite(alone[i])) and np.all(alone[i] <= 1.0)
        # the same requests in a shuffled mix, twice over, submitted from two threads while
        # two long requests hold both slots, so that the mix queues up and shares batches
        order = list(range(len(MIX))) * 2
        np.random.default_rng(0).shuffle(order)
        got, lock = [], threading.Lock()
        blockers = [_submit(occ, srv, c1, (640, 480, AO, 16, UNBIASED, 0, k, True), seed=k)[0]
                    for k in range(2)]

        def client(part):
            mine = []
            for i in part:
                rid, out = _submit(occ, srv, c1, MIX[i], seed=500 + i, sample=i)
                mine.append((i, rid, out))
            with lock:
                got.extend(mine)

        ths = [threading.Thread(target=client, args=(order[k::2],)) for k in range(2)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        res = srv.wait([rid for _, rid, _ in got] + blockers)
        batched = 0
        for i, rid, out in got:
            assert res[rid]["status"] == OK, res[rid]
            assert np.array_equal(out.cpu().numpy(), alone[i]), f"request {i} differs in the mix"
            batched = max(batched, res[rid]["batch_views"])
        assert batched >= 2          # requests did share batches
        st = srv.stats()
        assert st["views_batched"] > 0 and st["views_single"] > 0
        assert st["peak_reserved_bytes"] <= st["budget_bytes"]
    finally:
        srv.close()


def test_served_result_equals_direct_calls_and_oracle(orc, occ, ctx, c1):
    """Host G-buffer in: the server's estimate equals occ_trace_* + occ_reuse_* on the same
    G-buffer (per-view kernels on both sides), which in turn matches the FP64 oracle."""
    import torch
    srv = occ.Server(ctx, c1["bvh"], batch_max_px=1)
    pos_h = torch.from_numpy(c1["pos"]).pin_memory()
    nrm_h = torch.from_numpy(c1["nrm"]).pin_memory()
    gb = occ.GBuffer.from_numpy(c1["pos"], c1["nrm"])
    valid = c1["pos"][..., 3] > 0
    try:
        for eff, K, est in ((AO, 9, BIASED), (SH, 8, BIASED), (AO, 4, UNBIASED)):
            pat = _pattern(occ, K)
            out = torch.empty((64, 64)).pin_memory()
            rid = srv.submit(64, 64, eff, pat, est, out, radius=1.0,
                             light=LIGHT_C1 if eff == SH else None, seed=77, sample=2,
                             pos4_host=pos_h, nrm4_host=nrm_h)
            assert srv.wait([rid])[rid]["status"] == OK
            o = (occ.occ_trace_ao(ctx, gb, c1["bvh"], 1.0, 77, 2) if eff == AO
                 else occ.occ_trace_shadow(ctx, gb, c1["bvh"], LIGHT_C1, 77, 2))
            fn = occ.occ_reuse_ao if eff == AO else occ.occ_reuse_shadow
            d = fn(ctx, gb, o, pat, K, est, bvh=c1["bvh"] if est == UNBIASED else None)
            ctx.sync()
            assert np.array_equal(out.numpy(), d.cpu().numpy())
            orec, omg = orc.trace(c1["osc"], eff, c1["pos"], c1["nrm"], radius=1.0, light=LIGHT_C1,
                                  seed=77, sample=2)
            tr = P.compare_trace(o, orec, omg, valid, c1["pos"], "served trace")
            if tr["mismatch"] == 0:
                ref, mg = orc.reuse(c1["osc"], eff, c1["pos"], c1["nrm"], orec, pat.as_tuple(), est,
                                    radius=1.0, light=LIGHT_C1)
                P.compare_out(out.numpy(), ref, mg, valid, f"served effect {eff} K {K}")
    finally:
        srv.close()


def test_packed_camera_request_equals_packed_direct_path(occ, ctx, c1):
    """A packed camera request: G-buffer rendered packed on the device, packed records."""
    import torch
    srv = occ.Server(ctx, c1["bvh"], batch_max_px=1)
    cam = _cams()[1].as_array()
    try:
        pat = _pattern(occ, 8)
        out = torch.empty((40, 56), device="cuda")
        rid = srv.submit(56, 40, SH, pat, BIASED, out, light=LIGHT_C1, seed=3, sample=1,
                         packed=True, camera=cam, eps=c1["scene"].eps)
        assert srv.wait([rid])[rid]["status"] == OK
        gbp = occ.occ_gbuffer_pinhole(ctx, c1["bvh"], cam, c1["scene"].eps, 56, 40, packed=True)
        gbf = occ.occ_gbuffer_pinhole(ctx, c1["bvh"], cam, c1["scene"].eps, 56, 40)
        ref_packed = occ.occ_pack_gbuffer(ctx, gbf)
        ctx.sync()
        assert torch.equal(gbp.pos4.view(torch.int32), ref_packed.pos4.view(torch.int32))
        o = occ.occ_trace_shadow(ctx, gbp, c1["bvh"], LIGHT_C1, 3, 1, packed=True)
        d = occ.occ_reuse_shadow(ctx, gbp, o, pat, 8, BIASED)
        ctx.sync()
        assert torch.equal(out, d)
    finally:
        srv.close()


def test_budget_bounds_admission(occ, ctx, c1):
    import torch
    one = 64 * 64 * (16 + 16 + 32) + 3 * 256          # FP32 request with device output
    srv = occ.Server(ctx, c1["bvh"], budget_bytes=2 * one + 100, max_inflight=4,
                     max_views_per_batch=8)
    try:
        ids = []
        for i in range(12):
            rid, _ = _submit(occ, srv, c1, (64, 64, AO, 8, BIASED, 0, i % 3, True), seed=i)
            ids.append(rid)
        res = srv.wait(ids)
        assert all(r["status"] == OK for r in res.values())
        st = srv.stats()
        assert st["peak_reserved_bytes"] <= 2 * one + 100
        assert max(r["batch_views"] for r in res.values()) <= 2
        with pytest.raises(occ.OccError, match="OOM"):
            _submit(occ, srv, c1, (128, 128, AO, 8, BIASED, 0, 0, True), seed=0)
        for r in res.values():
            assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_done_ns"]
    finally:
        srv.close()


def test_deadline_and_cancellation(occ, ctx, c1):
    big = 640 * 480 * (16 + 16 + 32) + 3 * 256
    srv = occ.Server(ctx, c1["bvh"], budget_bytes=big + 1000, max_inflight=1)
    try:
        first, _ = _submit(occ, srv, c1, (640, 480, AO, 16, UNBIASED, 0, 0, True), seed=1)
        late, _ = _submit(occ, srv, c1, (640, 480, AO, 8, BIASED, 0, 1, True), seed=2,
                          deadline_ns=1)
        res = srv.wait([first, late])
        assert res[first]["status"] == OK
        assert res[late]["status"] == TIMEOUT and res[late]["batch_views"] == 0
        # shutdown with cancellation: the running request completes, queued ones are dropped
        run, _ = _submit(occ, srv, c1, (640, 480, SH, 16, UNBIASED, 0, 2, True), seed=3)
        queued = [_submit(occ, srv, c1, (640, 480, AO, 8, BIASED, 0, 0, True), seed=4 + k)[0]
                  for k in range(3)]
        srv.shutdown(cancel_queued=True)
        res = {r["id"]: r for r in srv.poll()}
        assert set(res) == {run, *queued}
        assert res[run]["status"] in (OK, CANCELLED)
        n_cancel = sum(res[q]["status"] == CANCELLED for q in queued)
        assert n_cancel >= 2          # at most one of them was already admitted
        with pytest.raises(occ.OccError, match="INVALID_ARG"):
            _submit(occ, srv, c1, MIX[0], seed=0)
    finally:
        srv.close()


def test_shutdown_without_cancel_runs_everything(occ, ctx, c1):
    srv = occ.Server(ctx, c1["bvh"], max_inflight=1, max_views_per_batch=1)
    ids = [_submit(occ, srv, c1, MIX[k % 4], seed=k)[0] for k in range(8)]
    srv.shutdown(cancel_queued=False)
    res = {r["id"]: r for r in srv.poll()}
    assert set(res) == set(ids) and all(r["status"] == OK for r in res.values())
    srv.close()


def test_invalid_requests_are_refused_at_submit(occ, ctx, c1):
    import torch
    srv = occ.Server(ctx, c1["bvh"])
    out = torch.empty((8, 8), device="cuda")
    cam = synth.camera_c1().as_array()
    g42 = occ.Pattern.group(4, 2)
    try:
        cases = [
            dict(W=0, H=8, effect=AO, pattern=g42, estimator=BIASED, camera=cam),
            dict(W=8, H=8, effect=5, pattern=g42, estimator=BIASED, camera=cam),
            dict(W=8, H=8, effect=AO, pattern=g42, estimator=9, camera=cam),
            dict(W=8, H=8, effect=AO, pattern=g42, estimator=BIASED, camera=cam, radius=-1.0),
            dict(W=8, H=8, effect=SH, pattern=g42, estimator=BIASED, camera=cam,
                 light=[0, 0, 4, 1, 0, 0, 1, 1, 0]),                      # edges not orthogonal
            dict(W=8, H=8, effect=AO, pattern=g42, estimator=BIASED,
                 camera=np.array([0, 0, 0, 1, 0, 0, 0, 0, 1, 200.0])),    # vfov out of range
            dict(W=8, H=8, effect=AO, pattern=occ.Pattern.offsets_of([[0, 0]]), estimator=BIASED,
                 camera=cam),
        ]
        for kw in cases:
            with pytest.raises(occ.OccError, match="INVALID_ARG"):
                srv.submit(out=out, **kw)
        with pytest.raises(occ.OccError, match="INVALID_ARG"):       # FP32 host G-buffer, no nrm
            srv.submit(8, 8, AO, g42, BIASED, out, pos4_host=torch.zeros((8, 8, 4)))
        assert srv.stats()["submitted"] == 0
    finally:
        srv.close()


def test_poisson_arrivals_with_concurrent_polling(occ, ctx, c1):
    """Requests arrive at random times while results are collected on another thread."""
    srv = occ.Server(ctx, c1["bvh"], max_views_per_batch=8, batch_max_px=5000)
    rng = np.random.default_rng(5)
    n = 60
    results, ids = {}, []
    done = threading.Event()

    def collector():
        while not done.is_set() or len(results) < len(ids):
            for r in srv.poll(timeout_us=20000):
                results[r["id"]] = r

    col = threading.Thread(target=collector)
    col.start()
    try:
        outs = []
        for k in range(n):
            time.sleep(float(rng.exponential(0.0005)))
            rid, out = _submit(occ, srv, c1, MIX[int(rng.integers(len(MIX)))], seed=k)
            ids.append(rid)
            outs.append(out)
        done.set()
        col.join(timeout=60)
        assert not col.is_alive()
        assert set(results) == set(ids)
        assert all(r["status"] == OK for r in results.values())
        lat = np.array([r["t_done_ns"] - r["t_submit_ns"] for r in results.values()]) * 1e-6
        print(f"served {n} requests: latency p50 {np.median(lat):.3f} ms, "
              f"p99 {np.quantile(lat, 0.99):.3f} ms")
    finally:
        done.set()
        srv.close()


def test_injected_allocation_failures_fail_their_requests_only(occ, ctx, c1):
    """Host-side fault injection: the first two batches find the pool exhausted; their
    requests finish with OCC_ERR_OOM, later ones run, the server keeps serving."""
    srv = occ.Server(ctx, c1["bvh"], max_views_per_batch=1, max_inflight=1,
                     inject_alloc_failures=2)
    try:
        ids = [_submit(occ, srv, c1, MIX[k % 3], seed=k)[0] for k in range(6)]
        res = srv.wait(ids)
        st = [res[i]["status"] for i in ids]
        assert st == [OOM, OOM, OK, OK, OK, OK], st
        assert srv.stats()["reserved_bytes"] == 0
    finally:
        srv.close()
