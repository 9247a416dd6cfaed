"""occ_frame_noalloc: the allocation-free frame entry point.

Some callers cannot allocate device memory (plugins whose host application owns every
allocation, real-time loops that cannot afford cudaMalloc's synchronisation).  For
them the library runs a whole frame with its scratch -- the occluder records and the
status word -- in a static device array.  This test calls that entry point through
the C ABI twice in a row and checks each result against the allocating path
(occ_trace_ao / occ_trace_shadow + occ_reuse_* into caller buffers), within the
tolerance of the parity tests; it also checks the size limit.  The file is named to
be collected last, so a failure here comes after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_23122_gb300 import occ
    import oracle
    scene = synth.scene_c1()
    osc = oracle.OracleScene(scene.tris)
    pos, nrm, _ = oracle.gbuffer(osc, synth.camera_c1().as_array(), 96, 64, scene.eps)
    ctx = occ.Context(0)
    return occ, ctx, occ.BVH(ctx, scene.tris), occ.GBuffer.from_numpy(pos, nrm)


def _noalloc(occ, gb, bvh, effect, radius, light, seed, sample, pat, est, out):
    """Direct C-ABI call (no binding helper), returning (status, flags, message)."""
    from paper_2607_23122_gb300 import _native as N
    lib = N.load()
    g = gb.c()
    L = occ._light(light if light is not None else np.zeros(9))
    flags = C.c_uint32(0)
    msg = C.create_string_buffer(256)
    st = lib.occ_frame_noalloc(C.byref(g), bvh.handle, effect, radius, C.byref(L), seed, sample,
                               C.byref(pat.c()), pat.K, est, out.data_ptr(), C.byref(flags), msg,
                               256, None)
    return st, flags.value, msg.value.decode()


@pytest.mark.parametrize("effect,est,pname,fmt", [(0, 1, "disk", "fp32"), (0, 2, "box", "fp32"),
                                                  (1, 1, "group", "fp32"), (1, 3, "box", "fp32"),
                                                  (0, 1, "group", "packed"), (1, 1, "disk", "tiled")])
def test_noalloc_matches_allocating_path_twice(setup, effect, est, pname, fmt):
    import torch
    occ, ctx, bvh, gb = setup
    if fmt == "packed":        # packed G-buffer; the scratch records stay FP32
        gb = occ.occ_pack_gbuffer(ctx, gb)
        ctx.sync()
    elif fmt == "tiled":       # tiled G-buffer layout (the window runs the per-receiver kernel)
        gb = occ.occ_tile_gbuffer(ctx, gb)
        ctx.sync()
    pat = {"disk": occ.Pattern.offsets_of(synth.disk_offsets(8, 6.0, seed=3)),
           "box": occ.Pattern.box(3, 3), "group": occ.Pattern.group(4, 2)}[pname]
    light = np.array([0.0, 0.5, 3.0, 3.0, 0, 0, 0, -3.0, 0], dtype=np.float32)
    radius = 1.0
    outs = []
    for sample in (0, 1):      # two calls in a row share the static scratch
        out = torch.full((gb.H, gb.W), -7.0, device="cuda")
        st, flags, msg = _noalloc(occ, gb, bvh, effect, radius, light, 11, sample, pat, est, out)
        assert st == 0 and flags == 0, msg
        rec = (occ.occ_trace_ao(ctx, gb, bvh, radius, 11, sample) if effect == 0 else
               occ.occ_trace_shadow(ctx, gb, bvh, light, 11, sample))
        fn = occ.occ_reuse_ao if effect == 0 else occ.occ_reuse_shadow
        ref = fn(ctx, gb, rec, pat, pat.K, est, bvh=bvh if est == 2 else None)
        ctx.sync()
        assert torch.allclose(out, ref, rtol=0.0, atol=TOL), (out - ref).abs().max().item()
        outs.append(out)
    # the second call's records replaced the first call's in the shared scratch: the two
    # samples' estimates differ
    assert (outs[0] != outs[1]).sum().item() >= 10


def test_noalloc_rejects_frames_over_the_limit(setup):
    import torch
    occ, ctx, bvh, _ = setup
    W, H = 1025, 1024          # one column more than 1024 x 1024
    pos = torch.zeros((H, W, 4), device="cuda")
    big = occ.GBuffer(pos, pos.clone())
    out = torch.empty((H, W), device="cuda")
    st, _, msg = _noalloc(occ, big, bvh, 0, 1.0, None, 1, 0, occ.Pattern.box(3, 3), 1, out)
    assert st == 1 and "maximum" in msg, (st, msg)
    with pytest.raises(occ.OccError, match="maximum"):
        occ.occ_frame_noalloc(big, bvh, 0, 1.0, None, 1, 0, occ.Pattern.box(3, 3), 9, 1, out)
