"""Python binding of the occlusion-point reuse library (include/occ.h).

Argument marshalling only: every step of the path runs in liboccreuse.so's CUDA
kernels.  PyTorch supplies device memory and streams; functions keep the C names.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _native as N
from ._native import (  # noqa: F401
    OCC_EFFECT_AO, OCC_EFFECT_SHADOW, OCC_EST_BIASED, OCC_EST_BOXMEAN, OCC_EST_LIGHT_UNBIASED,
    OCC_EST_NOREUSE, OCC_EST_UNBIASED, OCC_GB_FP32, OCC_GB_PACKED, OCC_LAYOUT_LINEAR,
    OCC_LAYOUT_TILED, OCC_PAT_BOX, OCC_PAT_GROUP, OCC_PAT_OFFSETS,
    OCC_PAT_RANDOM,
    OCC_REC_FP32, OCC_REC_PACKED, MAX_MEMBERS)


class OccError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{N.STATUS_NAMES.get(status, status)}: {message}")


def _stream_handle(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class Context:
    """An occ_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = N.load()
        self.device = device
        torch.cuda.set_device(device)
        torch.cuda.init()
        h = C.c_void_p()
        st = self.lib.occ_create(device, C.byref(h))
        if st != N.OCC_OK:
            raise OccError(st, f"occ_create(device={device}) failed")
        self.handle = h

    def check(self, st: int):
        if st != N.OCC_OK:
            msg = self.lib.occ_last_error(self.handle)
            raise OccError(st, msg.decode() if msg else "")

    def sync(self, stream=None):
        self.check(self.lib.occ_sync(self.handle, _stream_handle(stream)))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.occ_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def occ_create(device: int = 0) -> Context:
    return Context(device)


def occ_version() -> str:
    return N.load().occ_version().decode()


class BVH:
    """Device-resident 4-wide BVH built from float32 triangles [T, 3, 3]."""

    def __init__(self, ctx: Context, tris: np.ndarray):
        self.ctx = ctx
        tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 3, 3)
        h = C.c_void_p()
        ctx.check(ctx.lib.occ_bvh_build(ctx.handle, tris.ctypes.data, tris.shape[0], C.byref(h)))
        self.handle = h
        self.num_tris = tris.shape[0]

    @property
    def stats(self) -> dict:
        s = N.occ_bvh_stats()
        self.ctx.check(self.ctx.lib.occ_bvh_info(self.handle, C.byref(s)))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def free(self):
        if getattr(self, "handle", None) and self.ctx.handle:
            self.ctx.lib.occ_bvh_free(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def occ_bvh_build(ctx: Context, tris: np.ndarray) -> BVH:
    return BVH(ctx, tris)


def occ_debug_bvh_host(tris: np.ndarray):
    """The BVH builder alone on the host (no device): (nodes [N, 32] float32, triangles
    [T, 12] float32 in leaf order, depth); layouts as in include/occ.h."""
    lib = N.load()
    t = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
    T = t.shape[0]
    n, d = C.c_int64(0), C.c_int32(0)
    st = lib.occ_debug_bvh_host(t.ctypes.data, T, None, 0, None, 0, C.byref(n), C.byref(d))
    if st != 0:
        raise OccError(st, "host BVH build failed")
    nodes = np.empty((n.value, 32), dtype=np.float32)
    out = np.empty((T, 12), dtype=np.float32)
    st = lib.occ_debug_bvh_host(t.ctypes.data, T, nodes.ctypes.data, n.value, out.ctypes.data, T,
                                C.byref(n), C.byref(d))
    if st != 0:
        raise OccError(st, "host BVH build failed")
    return nodes, out, d.value


@dataclass
class GBuffer:
    """pos4 / nrm4: float32 CUDA tensors [H, W, 4] (see occ_gbuffer).  A packed G-buffer
    has only pos4 (the packed plane) and nrm4 = None.  A tiled G-buffer (OCC_LAYOUT_TILED,
    made by occ_tile_gbuffer) holds [ceil(H/8) * ceil(W/8), 64, 4] tensors and its size in
    `size` = (W, H)."""
    pos4: torch.Tensor
    nrm4: torch.Tensor | None = None
    layout: int = N.OCC_LAYOUT_LINEAR
    size: tuple | None = None

    @property
    def tiled(self) -> bool:
        return self.layout == N.OCC_LAYOUT_TILED

    @property
    def W(self) -> int:
        return int(self.size[0]) if self.tiled else int(self.pos4.shape[1])

    @property
    def H(self) -> int:
        return int(self.size[1]) if self.tiled else int(self.pos4.shape[0])

    @property
    def packed(self) -> bool:
        return self.nrm4 is None

    @property
    def pitch(self) -> int:
        """Row pitch of the planes in pixels (the tensors may be windows of wider ones); 0 for
        a tiled G-buffer."""
        return 0 if self.tiled else int(self.pos4.stride(0)) // 4

    def c(self) -> N.occ_gbuffer:
        for t in (self.pos4,) if self.packed else (self.pos4, self.nrm4):
            if self.tiled:
                n = ((self.W + 7) // 8) * ((self.H + 7) // 8)
                if not (t.is_cuda and t.dtype == torch.float32 and tuple(t.shape) == (n, 64, 4)
                        and t.is_contiguous()):
                    raise ValueError("tiled G-buffer tensors must be contiguous float32 CUDA "
                                     "[ceil(H/8) * ceil(W/8), 64, 4]")
            elif not (t.is_cuda and t.dtype == torch.float32 and tuple(t.shape) == (self.H, self.W, 4)
                      and t.stride(2) == 1 and t.stride(1) == 4 and t.stride(0) % 4 == 0
                      and t.stride(0) // 4 == self.pitch and self.pitch >= self.W):
                raise ValueError("G-buffer tensors must be float32 CUDA [H, W, 4] with contiguous "
                                 "rows and the same row pitch")
        return N.occ_gbuffer(W=self.W, H=self.H, pos4=self.pos4.data_ptr(),
                             nrm4=None if self.packed else self.nrm4.data_ptr(),
                             format=N.OCC_GB_PACKED if self.packed else N.OCC_GB_FP32,
                             layout=self.layout, pitch_px=self.pitch)

    @staticmethod
    def from_numpy(pos4: np.ndarray, nrm4: np.ndarray, device="cuda") -> "GBuffer":
        return GBuffer(torch.from_numpy(np.ascontiguousarray(pos4, dtype=np.float32)).to(device),
                       torch.from_numpy(np.ascontiguousarray(nrm4, dtype=np.float32)).to(device))


@dataclass
class Occluders:
    """Occluder records: data is a float32 CUDA tensor [2, H, W, 4] (two FP32 planes) or
    [1, H, W, 4] (the packed plane, 16 bytes per pixel)."""
    data: torch.Tensor
    meta: N.occ_occluders = field(default_factory=N.occ_occluders)

    @staticmethod
    def empty(H: int, W: int, device="cuda", packed: bool = False) -> "Occluders":
        o = Occluders(torch.empty((1 if packed else 2, H, W, 4), dtype=torch.float32,
                                  device=device))
        o.meta.W, o.meta.H = W, H
        o.meta.format = N.OCC_REC_PACKED if packed else N.OCC_REC_FP32
        o.meta.data = o.data.data_ptr()
        return o

    @staticmethod
    def from_packed(plane: np.ndarray, effect: int, radius: float = 0.0, light=None,
                    device="cuda", sample: int = 0) -> "Occluders":
        """Packed records prepared elsewhere: [H, W, 4] float32 view of the 16-byte records."""
        H, W = plane.shape[:2]
        o = Occluders.empty(H, W, device, packed=True)
        o.data[0].copy_(torch.from_numpy(np.ascontiguousarray(plane, dtype=np.float32)))
        o.meta.effect = effect
        o.meta.radius = radius
        o.meta.sample = sample
        if light is not None:
            o.meta.light = _light(light)
        return o

    @property
    def packed(self) -> bool:
        return self.meta.format == N.OCC_REC_PACKED

    @staticmethod
    def from_numpy(rec0: np.ndarray, rec1: np.ndarray, effect: int, radius: float = 0.0,
                   light=None, device="cuda", sample: int = 0) -> "Occluders":
        """Records prepared elsewhere (e.g. test inputs): planes [H, W, 4] float32; `sample`
        is the records' sample index (random patterns draw their offsets with it)."""
        H, W = rec0.shape[:2]
        o = Occluders.empty(H, W, device)
        o.data[0].copy_(torch.from_numpy(np.ascontiguousarray(rec0, dtype=np.float32)))
        o.data[1].copy_(torch.from_numpy(np.ascontiguousarray(rec1, dtype=np.float32)))
        o.meta.effect = effect
        o.meta.radius = radius
        o.meta.sample = sample
        if light is not None:
            o.meta.light = _light(light)
        return o

    def c(self) -> N.occ_occluders:
        self.meta.data = self.data.data_ptr()
        return self.meta

    @property
    def tri(self) -> torch.Tensor:
        return self.data[0, ..., 3].contiguous().view(torch.int32)


def _light(light) -> N.occ_rect_light:
    v = np.asarray(light, dtype=np.float32).reshape(9)
    L = N.occ_rect_light()
    L.c[:] = v[0:3].tolist()
    L.eu[:] = v[3:6].tolist()
    L.ev[:] = v[6:9].tolist()
    return L


class Pattern:
    """Neighbour pattern N_i: group blocks, a centred box, shared offsets, or offsets drawn
    per receiver and sample in a disk (random)."""

    def __init__(self, kind: int, gw: int = 1, gh: int = 1, offsets=None, n_random: int = 0,
                 radius_px: int = 0, seed: int = 0):
        self.kind, self.gw, self.gh = int(kind), int(gw), int(gh)
        off = np.zeros((0, 2), dtype=np.int32) if offsets is None else offsets
        self.offsets = np.ascontiguousarray(np.asarray(off, dtype=np.int32).reshape(-1, 2))
        self.n_random, self.radius_px, self.seed = int(n_random), int(radius_px), int(seed)
        n_off = self.n_random if self.kind == N.OCC_PAT_RANDOM else self.offsets.shape[0]
        self._c = N.occ_pattern(self.kind, self.gw, self.gh, n_off,
                                self.offsets.ctypes.data_as(C.POINTER(C.c_int32)),
                                self.radius_px, self.seed)

    @staticmethod
    def group(gw: int, gh: int) -> "Pattern":
        return Pattern(N.OCC_PAT_GROUP, gw, gh)

    @staticmethod
    def box(gw: int, gh: int) -> "Pattern":
        return Pattern(N.OCC_PAT_BOX, gw, gh)

    @staticmethod
    def offsets_of(off) -> "Pattern":
        return Pattern(N.OCC_PAT_OFFSETS, 1, 1, off)

    @staticmethod
    def random(K: int, radius_px: int, seed: int) -> "Pattern":
        """The receiver plus K - 1 offsets drawn per receiver and sample in a disk."""
        return Pattern(N.OCC_PAT_RANDOM, n_random=K - 1, radius_px=radius_px, seed=seed)

    @property
    def K(self) -> int:
        if self.kind == N.OCC_PAT_OFFSETS:
            return self.offsets.shape[0] + 1
        if self.kind == N.OCC_PAT_RANDOM:
            return self.n_random + 1
        return self.gw * self.gh

    def as_tuple(self):
        """(kind, gw, gh, offsets), or (random kind, radius, n_offsets, seed) -- the form the
        oracle takes."""
        if self.kind == N.OCC_PAT_RANDOM:
            return (self.kind, self.radius_px, self.n_random, self.seed)
        return (self.kind, self.gw, self.gh, self.offsets if self.offsets.size else None)

    def c(self) -> N.occ_pattern:
        return self._c


def occ_gbuffer_pinhole(ctx: Context, bvh: BVH, camera, eps: float, W: int, H: int,
                        stream=None, packed: bool = False) -> GBuffer:
    cam = np.ascontiguousarray(camera, dtype=np.float32).reshape(10)
    dev = torch.device("cuda", ctx.device)
    gb = GBuffer(torch.empty((H, W, 4), dtype=torch.float32, device=dev),
                 None if packed else torch.empty((H, W, 4), dtype=torch.float32, device=dev))
    ctx.check(ctx.lib.occ_gbuffer_pinhole(ctx.handle, bvh.handle, cam.ctypes.data, float(eps), W, H,
                                          gb.pos4.data_ptr(), None if packed else gb.nrm4.data_ptr(),
                                          _stream_handle(stream)))
    return gb


def occ_pack_gbuffer(ctx: Context, gb: GBuffer, stream=None) -> GBuffer:
    """FP32 G-buffer -> packed G-buffer (16 bytes per pixel)."""
    out = torch.empty((gb.H, gb.W, 4), dtype=torch.float32, device=gb.pos4.device)
    g = gb.c()
    ctx.check(ctx.lib.occ_pack_gbuffer(ctx.handle, C.byref(g), out.data_ptr(),
                                       _stream_handle(stream)))
    return GBuffer(out, None)


def occ_tile_gbuffer(ctx: Context, gb: GBuffer, stream=None) -> GBuffer:
    """The same G-buffer in the tiled layout (8 x 8 tiles, Morton order inside a tile)."""
    n = ((gb.W + 7) // 8) * ((gb.H + 7) // 8)
    dev = gb.pos4.device
    pos = torch.empty((n, 64, 4), dtype=torch.float32, device=dev)
    nrm = None if gb.packed else torch.empty((n, 64, 4), dtype=torch.float32, device=dev)
    g = gb.c()
    ctx.check(ctx.lib.occ_tile_gbuffer(ctx.handle, C.byref(g), pos.data_ptr(),
                                       None if nrm is None else nrm.data_ptr(),
                                       _stream_handle(stream)))
    return GBuffer(pos, nrm, layout=N.OCC_LAYOUT_TILED, size=(gb.W, gb.H))


def occ_trace_ao(ctx: Context, gb: GBuffer, bvh: BVH, radius: float, seed: int, sample: int,
                 out: Occluders | None = None, stream=None, packed: bool = False) -> Occluders:
    out = out or Occluders.empty(gb.H, gb.W, gb.pos4.device, packed=packed)
    g = gb.c()
    ctx.check(ctx.lib.occ_trace_ao(ctx.handle, C.byref(g), bvh.handle, float(radius), int(seed),
                                   int(sample), C.byref(out.c()), _stream_handle(stream)))
    return out


def occ_trace_shadow(ctx: Context, gb: GBuffer, bvh: BVH, light, seed: int, sample: int,
                     out: Occluders | None = None, stream=None, packed: bool = False) -> Occluders:
    out = out or Occluders.empty(gb.H, gb.W, gb.pos4.device, packed=packed)
    g = gb.c()
    L = _light(light)
    ctx.check(ctx.lib.occ_trace_shadow(ctx.handle, C.byref(g), bvh.handle, C.byref(L), int(seed),
                                       int(sample), C.byref(out.c()), _stream_handle(stream)))
    return out


def _reuse(fn, ctx, gb, occ, pattern, K, estimator, bvh, out, stream):
    if out is None:
        out = torch.empty((gb.H, gb.W), dtype=torch.float32, device=gb.pos4.device)
    g = gb.c()
    ctx.check(fn(ctx.handle, C.byref(g), C.byref(occ.c()), C.byref(pattern.c()), int(K),
                 int(estimator), bvh.handle if bvh is not None else None, out.data_ptr(),
                 _stream_handle(stream)))
    return out


def occ_reuse_ao(ctx: Context, gb: GBuffer, occ: Occluders, pattern: Pattern, K: int,
                 estimator: int, bvh: BVH | None = None, out: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    return _reuse(ctx.lib.occ_reuse_ao, ctx, gb, occ, pattern, K, estimator, bvh, out, stream)


def occ_reuse_shadow(ctx: Context, gb: GBuffer, occ: Occluders, pattern: Pattern, K: int,
                     estimator: int, bvh: BVH | None = None, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    return _reuse(ctx.lib.occ_reuse_shadow, ctx, gb, occ, pattern, K, estimator, bvh, out, stream)


def occ_trace_reuse_ao(ctx: Context, gb: GBuffer, bvh: BVH, radius: float, seed: int,
                       sample: int, pattern: Pattern, K: int, estimator: int,
                       rec: Occluders | None = None, out: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
    """Steps 1-3 in one kernel for a group pattern (occ_trace_reuse_ao); `rec`, when given,
    also receives the step-1 records."""
    if out is None:
        out = torch.empty((gb.H, gb.W), dtype=torch.float32, device=gb.pos4.device)
    g = gb.c()
    ctx.check(ctx.lib.occ_trace_reuse_ao(ctx.handle, C.byref(g), bvh.handle, float(radius),
                                         int(seed), int(sample), C.byref(pattern.c()), int(K),
                                         int(estimator), C.byref(rec.c()) if rec is not None else None,
                                         out.data_ptr(), _stream_handle(stream)))
    return out


def occ_trace_reuse_shadow(ctx: Context, gb: GBuffer, bvh: BVH, light, seed: int, sample: int,
                           pattern: Pattern, K: int, estimator: int, rec: Occluders | None = None,
                           out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Shadow counterpart of occ_trace_reuse_ao."""
    if out is None:
        out = torch.empty((gb.H, gb.W), dtype=torch.float32, device=gb.pos4.device)
    g = gb.c()
    L = _light(light)
    ctx.check(ctx.lib.occ_trace_reuse_shadow(ctx.handle, C.byref(g), bvh.handle, C.byref(L),
                                             int(seed), int(sample), C.byref(pattern.c()), int(K),
                                             int(estimator),
                                             C.byref(rec.c()) if rec is not None else None,
                                             out.data_ptr(), _stream_handle(stream)))
    return out


def occ_shadow_lights(ctx: Context, gb: GBuffer, bvh: BVH, lights, weights, seed: int,
                      sample: int, pattern: Pattern, estimator: int, packed: bool = False,
                      stream=None):
    """out = sum_l weights[l] * V_l over several lights (occ_shadow_lights); returns
    (out [H, W], vis [n_lights, H, W], records)."""
    lights = [np.asarray(l, dtype=np.float32).reshape(9) for l in lights]
    n = len(lights)
    dev = gb.pos4.device
    recs = [Occluders.empty(gb.H, gb.W, dev, packed=packed) for _ in range(n)]
    arr_l = (N.occ_rect_light * n)(*[_light(l) for l in lights])
    arr_r = (N.occ_occluders * n)(*[r.c() for r in recs])
    w = np.ascontiguousarray(weights, dtype=np.float32).reshape(n)
    vis = torch.empty((n, gb.H, gb.W), dtype=torch.float32, device=dev)
    out = torch.empty((gb.H, gb.W), dtype=torch.float32, device=dev)
    g = gb.c()
    ctx.check(ctx.lib.occ_shadow_lights(ctx.handle, C.byref(g), bvh.handle, arr_l, w.ctypes.data, n,
                                        seed, sample, C.byref(pattern.c()), pattern.K, estimator,
                                        arr_r, vis.data_ptr(), out.data_ptr(),
                                        _stream_handle(stream)))
    for r, m in zip(recs, arr_r):
        r.meta = m
    return out, vis, recs


def occ_frame_host(ctx: Context, bvh: BVH, effect: int, pos4_host: torch.Tensor,
                   nrm4_host: torch.Tensor, radius: float, light, seed: int, sample: int,
                   pattern: Pattern, K: int, estimator: int, out_host: torch.Tensor,
                   stream=None) -> torch.Tensor:
    """Whole frame from host tensors (pinned recommended) to a host estimate [H, W]."""
    H, W = int(pos4_host.shape[0]), int(pos4_host.shape[1])
    L = _light(light if light is not None else np.zeros(9))
    ctx.check(ctx.lib.occ_frame_host(ctx.handle, bvh.handle, int(effect), pos4_host.data_ptr(),
                                     nrm4_host.data_ptr(), W, H, float(radius), C.byref(L),
                                     int(seed), int(sample), C.byref(pattern.c()), int(K),
                                     int(estimator), out_host.data_ptr(), _stream_handle(stream)))
    return out_host


def occ_frame_host_async(ctx: Context, bvh: BVH, effect: int, pos4_host: torch.Tensor,
                         nrm4_host: torch.Tensor, radius: float, light, seed: int, sample: int,
                         pattern: Pattern, K: int, estimator: int, out_host: torch.Tensor,
                         stream=None) -> torch.Tensor:
    """occ_frame_host without the wait: out_host is valid once `stream` has completed
    (ctx.sync(stream)); one frame in flight per context."""
    H, W = int(pos4_host.shape[0]), int(pos4_host.shape[1])
    L = _light(light if light is not None else np.zeros(9))
    ctx.check(ctx.lib.occ_frame_host_async(ctx.handle, bvh.handle, int(effect),
                                           pos4_host.data_ptr(), nrm4_host.data_ptr(), W, H,
                                           float(radius), C.byref(L), int(seed), int(sample),
                                           C.byref(pattern.c()), int(K), int(estimator),
                                           out_host.data_ptr(), _stream_handle(stream)))
    return out_host


NOALLOC_MAX_PIXELS = 1 << 20


def occ_frame_noalloc(gb: GBuffer, bvh: BVH, effect: int, radius: float, light, seed: int,
                      sample: int, pattern: Pattern, K: int, estimator: int, out: torch.Tensor,
                      check: bool = True, stream=None) -> torch.Tensor:
    """One frame (trace + reuse) into `out` with no device allocation (see occ.h).

    For callers that cannot allocate device memory; frames up to NOALLOC_MAX_PIXELS.
    Records live in a library-static array shared by all calls, so calls must not
    overlap on the GPU.  With check=True the call waits for the stream and raises
    on device-check flags.
    """
    lib = N.load()
    g = gb.c()
    L = _light(light if light is not None else np.zeros(9))
    flags = C.c_uint32(0)
    msg = C.create_string_buffer(512)
    st = lib.occ_frame_noalloc(C.byref(g), bvh.handle, int(effect), float(radius), C.byref(L),
                               int(seed), int(sample), C.byref(pattern.c()), int(K),
                               int(estimator), out.data_ptr(), C.byref(flags) if check else None,
                               msg, 512, _stream_handle(stream))
    if st != N.OCC_OK:
        raise OccError(st, msg.value.decode())
    return out


def occ_debug_closest_hit(ctx: Context, bvh: BVH, o, d, tmax, any_hit: bool = False,
                          stream=None):
    """(tri [n] int32, t [n] float32) of arbitrary rays (occ_debug_closest_hit)."""
    o = np.asarray(o, dtype=np.float32).reshape(-1, 3)
    d = np.asarray(d, dtype=np.float32).reshape(-1, 3)
    n = o.shape[0]
    rays = np.zeros((n, 8), dtype=np.float32)
    rays[:, :3], rays[:, 3], rays[:, 4:7] = o, np.broadcast_to(np.asarray(tmax, np.float32), (n,)), d
    dev = torch.device("cuda", ctx.device)
    r = torch.from_numpy(rays).to(dev)
    tri = torch.empty(n, dtype=torch.int32, device=dev)
    t = torch.empty(n, dtype=torch.float32, device=dev)
    ctx.check(ctx.lib.occ_debug_closest_hit(ctx.handle, bvh.handle, r.data_ptr(), n, int(any_hit),
                                            tri.data_ptr(), t.data_ptr(), _stream_handle(stream)))
    ctx.sync(stream)
    return tri.cpu().numpy(), t.cpu().numpy()


def occ_debug_fp32_peak(ctx: Context, paired: bool, iters: int, blocks: int, sink: torch.Tensor,
                        stream=None) -> float:
    """Launches the FP32 throughput probe on `stream`; returns the launch's FLOP count."""
    assert sink.dtype == torch.float32 and sink.is_cuda and sink.numel() >= blocks * 256
    flop = C.c_double()
    ctx.check(ctx.lib.occ_debug_fp32_peak(ctx.handle, int(bool(paired)), int(iters), int(blocks),
                                          sink.data_ptr(), C.byref(flop), _stream_handle(stream)))
    return float(flop.value)


def occ_debug_stream_ceiling(ctx: Context, gb: GBuffer, occ: Occluders, out: torch.Tensor,
                             stream=None):
    """Launches the group kernel's streaming-ceiling probe (FP32 formats) on `stream`."""
    g = gb.c()
    ctx.check(ctx.lib.occ_debug_stream_ceiling(ctx.handle, C.byref(g), C.byref(occ.c()),
                                               out.data_ptr(), _stream_handle(stream)))


def occ_debug_bvh_counters(ctx: Context, bvh: BVH, reset: bool = True) -> dict:
    """Traversal counters of the instrumented library since the last reset."""
    out = (C.c_uint64 * 5)()
    ctx.check(ctx.lib.occ_debug_bvh_counters(ctx.handle, bvh.handle, int(bool(reset)), out))
    return {"node_visits": int(out[0]), "triangle_tests": int(out[1]),
            "distinct_nodes": int(out[2]), "distinct_triangles": int(out[3]),
            "distinct_bytes": int(out[4])}


def occ_debug_wait_timeout(ctx: Context, spins: int = 1000, stream=None):
    ctx.check(ctx.lib.occ_debug_wait_timeout(ctx.handle, int(spins), _stream_handle(stream)))


def occ_debug_philox(ctx: Context, ctr_key: np.ndarray, stream=None) -> np.ndarray:
    """Philox4x32-10 of rows (c0, c1, c2, c3, k0, k1) -> [n, 4] uint32 (synchronous)."""
    a = np.ascontiguousarray(ctr_key, dtype=np.uint32).reshape(-1, 6)
    dev = torch.device("cuda", ctx.device)
    inp = torch.from_numpy(a.view(np.int32)).to(dev)
    out = torch.empty((a.shape[0], 4), dtype=torch.int32, device=dev)
    ctx.check(ctx.lib.occ_debug_philox(ctx.handle, inp.data_ptr(), a.shape[0], out.data_ptr(),
                                       _stream_handle(stream)))
    ctx.sync(stream)
    return out.cpu().numpy().view(np.uint32)


def occ_debug_rays(ctx: Context, gb: GBuffer, effect: int, radius: float, light, seed: int,
                   sample: int, stream=None) -> torch.Tensor:
    out = torch.empty((gb.H, gb.W, 4), dtype=torch.float32, device=gb.pos4.device)
    g = gb.c()
    L = _light(light if light is not None else np.zeros(9))
    ctx.check(ctx.lib.occ_debug_rays(ctx.handle, C.byref(g), int(effect), float(radius), C.byref(L),
                                     int(seed), int(sample), out.data_ptr(),
                                     _stream_handle(stream)))
    return out


def occ_debug_mis(ctx: Context, gb: GBuffer, occ: Occluders, pattern: Pattern, K: int,
                  estimator: int, pix, bvh: BVH | None = None):
    """(members [n, 64] int32, weights [n, 64, 64] float32) for receivers `pix`."""
    pix = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1)
    n = pix.shape[0]
    mem = np.zeros((n, N.MAX_MEMBERS), dtype=np.int32)
    w = np.zeros((n, N.MAX_MEMBERS, N.MAX_MEMBERS), dtype=np.float32)
    g = gb.c()
    ctx.check(ctx.lib.occ_debug_mis(ctx.handle, C.byref(g), C.byref(occ.c()), C.byref(pattern.c()),
                                    int(K), int(estimator), bvh.handle if bvh is not None else None,
                                    pix.ctypes.data, n, mem.ctypes.data, w.ctypes.data))
    return mem, w


# ------------------------------------------------------------------------------------
# Batched frames, captured batches, tuning
# ------------------------------------------------------------------------------------

@dataclass
class View:
    """One view of a batched frame (see occ_view)."""
    gb: GBuffer
    rec: Occluders
    out: torch.Tensor
    effect: int = OCC_EFFECT_AO
    radius: float = 0.5
    light: object = None
    seed: int = 0
    sample: int = 0
    pattern: Pattern = None
    estimator: int = OCC_EST_BIASED

    def c(self) -> N.occ_view:
        v = N.occ_view()
        v.gb = self.gb.c()
        v.rec = self.rec.c()
        v.effect = self.effect
        v.radius = self.radius
        v.light = _light(self.light if self.light is not None else np.zeros(9))
        v.seed = self.seed
        v.sample = self.sample
        v.pattern = self.pattern.c()
        v.K = self.pattern.K
        v.estimator = self.estimator
        v.out = self.out.data_ptr()
        return v


def _views_array(views):
    arr = (N.occ_view * len(views))()
    for i, v in enumerate(views):
        arr[i] = v.c()
    return arr


def _copy_back(arr, views):
    for i, v in enumerate(views):
        v.rec.meta = arr[i].rec


def occ_frame_batch(ctx: Context, bvh: BVH, views: list, stream=None):
    """Trace and reuse every view in one persistent launch pair (occ_frame_batch)."""
    arr = _views_array(views)
    ctx.check(ctx.lib.occ_frame_batch(ctx.handle, bvh.handle, arr, len(views),
                                      _stream_handle(stream)))
    _copy_back(arr, views)


class Batch:
    """A batched frame captured as a CUDA graph; replay() runs it with new seeds/samples."""

    def __init__(self, ctx: Context, bvh: BVH, views: list):
        self.ctx, self.views = ctx, views
        arr = _views_array(views)
        h = C.c_void_p()
        ctx.check(ctx.lib.occ_batch_capture(ctx.handle, bvh.handle, arr, len(views), C.byref(h)))
        _copy_back(arr, views)
        self.handle = h

    def replay(self, seeds, samples, stream=None):
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        sm = np.ascontiguousarray(samples, dtype=np.uint32)
        assert sd.shape[0] == len(self.views) and sm.shape[0] == len(self.views)
        self.ctx.check(self.ctx.lib.occ_batch_launch(self.ctx.handle, self.handle, sd.ctypes.data,
                                                     sm.ctypes.data, _stream_handle(stream)))

    def free(self):
        if getattr(self, "handle", None):
            self.ctx.lib.occ_batch_free(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def occ_set_tuning(ctx: Context, reuse_tile_rows: int = 0, reuse_window_path: int = 0,
                   batch_ctas_per_sm: int = 0, fused_ao_path: int = 0, group_prefetch: int = 0,
                   trace_path: int = 0, trace_ctas_per_sm: int = 0, trace_refill: int = 0,
                   trace_order: int = 0):
    t = N.occ_tuning(reuse_tile_rows, reuse_window_path, batch_ctas_per_sm, fused_ao_path,
                     group_prefetch, trace_path, trace_ctas_per_sm, trace_refill, trace_order)
    ctx.check(ctx.lib.occ_set_tuning(ctx.handle, C.byref(t)))


def occ_get_tuning(ctx: Context) -> dict:
    t = N.occ_tuning()
    ctx.check(ctx.lib.occ_get_tuning(ctx.handle, C.byref(t)))
    return {f: getattr(t, f) for f, _ in t._fields_}


# --------------------------------------------------------------------------------------
# Serving loop (include/occ_serve.h)
# --------------------------------------------------------------------------------------

class Scheduler:
    """The admission scheduler alone (host only; occ_sched_*)."""

    def __init__(self, budget_bytes: int, max_views_per_batch: int = 64, max_inflight: int = 2,
                 max_queued: int = 4096):
        self.lib = N.load()
        cfg = N.occ_sched_config(budget_bytes, max_views_per_batch, max_inflight, max_queued)
        h = C.c_void_p()
        st = self.lib.occ_sched_create(C.byref(cfg), C.byref(h))
        if st != N.OCC_OK:
            raise OccError(st, "occ_sched_create: invalid configuration")
        self.handle = h
        self.cap = max_views_per_batch

    def submit(self, id: int, nbytes: int, now_ns: int, deadline_ns: int = 0) -> int:
        """Returns the status (0 = queued)."""
        return self.lib.occ_sched_submit(self.handle, id, nbytes, now_ns, deadline_ns)

    def next(self, now_ns: int, exp_cap: int = 256):
        """(slot or -1, admitted ids, expired ids)."""
        ids = (C.c_uint64 * self.cap)()
        exp = (C.c_uint64 * max(1, exp_cap))()
        n, slot, ne = C.c_int32(), C.c_int32(), C.c_int32()
        st = self.lib.occ_sched_next(self.handle, now_ns, ids, self.cap, C.byref(n), C.byref(slot),
                                     exp, exp_cap, C.byref(ne))
        if st != N.OCC_OK:
            raise OccError(st, "occ_sched_next")
        return slot.value, list(ids[:n.value]), list(exp[:ne.value])

    def complete(self, slot: int) -> int:
        return self.lib.occ_sched_complete(self.handle, slot)

    def drain(self) -> list:
        out = []
        buf = (C.c_uint64 * 64)()
        n = C.c_int32(64)
        while n.value == 64:
            self.lib.occ_sched_drain(self.handle, buf, 64, C.byref(n))
            out += list(buf[:n.value])
        return out

    def stats(self) -> dict:
        s = N.occ_sched_stats()
        self.lib.occ_sched_get_stats(self.handle, C.byref(s))
        return {f: getattr(s, f) for f, _ in s._fields_}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.occ_sched_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """A serving loop on ctx's device for one resident scene (occ_server_*).

    submit() takes one frame (camera or host G-buffer in; pinned host or device tensor out)
    and returns its id; poll() returns finished results as dicts with the server's own
    timestamps (ns since the server started)."""

    def __init__(self, ctx: Context, bvh: BVH, budget_bytes: int = 0, max_views_per_batch: int = 0,
                 max_inflight: int = 0, max_queued: int = 0, poll_us: int = 0,
                 batch_max_px: int = 0, batch_window_us: int = 0,
                 inject_alloc_failures: int = 0):
        self.ctx, self.bvh = ctx, bvh          # the BVH must outlive the server
        cfg = N.occ_server_config(budget_bytes, max_views_per_batch, max_inflight, max_queued,
                                  poll_us, batch_max_px, batch_window_us, inject_alloc_failures, 0)
        h = C.c_void_p()
        ctx.check(ctx.lib.occ_server_create(ctx.handle, bvh.handle, C.byref(cfg), C.byref(h)))
        self.handle = h
        self._keep = {}                        # id -> objects the request points into

    def submit(self, W: int, H: int, effect: int, pattern: Pattern, estimator: int, out,
               radius: float = 0.5, light=None, seed: int = 0, sample: int = 0,
               packed: bool = False, camera=None, eps: float = 0.0, pos4_host=None,
               nrm4_host=None, deadline_ns: int = 0) -> int:
        r = N.occ_request()
        r.W, r.H, r.effect, r.radius = W, H, effect, radius
        r.light = _light(light if light is not None else np.zeros(9))
        r.seed, r.sample = seed, sample
        r.pattern = pattern.c()
        r.K, r.estimator, r.packed = pattern.K, estimator, int(packed)
        if camera is not None:
            r.camera[:] = [float(v) for v in np.asarray(camera, dtype=np.float32).reshape(10)]
        r.eps = eps
        keep = [pattern]
        if pos4_host is not None:
            r.pos4_host = pos4_host.data_ptr()
            keep.append(pos4_host)
            if nrm4_host is not None:
                r.nrm4_host = nrm4_host.data_ptr()
                keep.append(nrm4_host)
        if out.is_cuda:
            r.out_device = out.data_ptr()
        else:
            r.out_host = out.data_ptr()
        keep.append(out)
        r.deadline_ns = deadline_ns
        rid = C.c_uint64()
        msg = C.create_string_buffer(256)
        st = self.ctx.lib.occ_server_submit(self.handle, C.byref(r), C.byref(rid), msg, 256)
        if st != N.OCC_OK:
            raise OccError(st, msg.value.decode(errors="replace"))
        self._keep[rid.value] = keep
        return rid.value

    def poll(self, max_results: int = 256, timeout_us: int = 0) -> list:
        buf = (N.occ_result * max_results)()
        n = C.c_int32()
        self.ctx.check(self.ctx.lib.occ_server_poll(self.handle, buf, max_results, timeout_us,
                                                    C.byref(n)))
        out = []
        for i in range(n.value):
            r = buf[i]
            self._keep.pop(r.id, None)
            out.append({"id": r.id, "status": r.status, "batch_views": r.batch_views,
                        "t_submit_ns": r.t_submit_ns, "t_admit_ns": r.t_admit_ns,
                        "t_done_ns": r.t_done_ns})
        return out

    def wait(self, ids, timeout_s: float = 60.0) -> dict:
        """Polls until every id in `ids` finished; returns {id: result}."""
        import time
        want, got = set(ids), {}
        end = time.monotonic() + timeout_s
        while want - got.keys():
            left = end - time.monotonic()
            if left <= 0:
                raise TimeoutError(f"{len(want - got.keys())} requests still running")
            for r in self.poll(timeout_us=int(min(left, 0.5) * 1e6)):
                got[r["id"]] = r
        return {i: got[i] for i in ids}

    def stats(self) -> dict:
        s = N.occ_server_stats()
        self.ctx.check(self.ctx.lib.occ_server_get_stats(self.handle, C.byref(s)))
        d = {f: getattr(s.sched, f) for f, _ in s.sched._fields_}
        d.update({f: getattr(s, f) for f, _ in s._fields_ if f != "sched"})
        return d

    def shutdown(self, cancel_queued: bool = False):
        """Stops accepting work; waits for the worker (results stay pollable)."""
        self.ctx.check(self.ctx.lib.occ_server_shutdown(self.handle, int(cancel_queued)))

    def close(self, cancel_queued: bool = False):
        if getattr(self, "handle", None):
            self.ctx.lib.occ_server_destroy(self.handle, int(cancel_queued))
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
