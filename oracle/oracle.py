"""ctypes front end of the FP64 C oracle (``occ_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It never touches the
CUDA library, and the CUDA library never touches it.

Every function takes NumPy arrays of the seeded input data (float32 triangles,
float32 G-buffers, float32 lights) and returns float64 results.  The oracle
parts, and the passages of the paper they follow, are listed in the header of
``occ_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "occ_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libocc_oracle.so")
_lock = threading.Lock()
_lib = None

EFFECT_AO, EFFECT_SHADOW = 0, 1
PAT_GROUP, PAT_BOX, PAT_OFFSETS, PAT_RANDOM = 0, 1, 2, 3
EST_NOREUSE, EST_BIASED, EST_UNBIASED, EST_BOXMEAN = 0, 1, 2, 3
EST_LIGHT_UNBIASED = 4       # shadows: unbiased light-sample reuse (Light(N U), Sec. 6.2)
STREAM_AO, STREAM_SHADOW = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc: -O2, OpenMP, no fast-math, no FP contraction."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unknown-pragmas", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _P(dt):
    return np.ctypeslib.ndpointer(dtype=dt, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        L = C.CDLL(build())
        f32, f64, i32, i64, u32 = _P(np.float32), _P(np.float64), _P(np.int32), _P(np.int64), _P(np.uint32)
        vp = C.c_void_p
        L.orc_philox4x32_10.argtypes = [u32, u32, u32]
        L.orc_uniform_pair.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, f64]
        L.orc_scene_create.argtypes = [f32, C.c_int64]
        L.orc_scene_create.restype = vp
        L.orc_scene_destroy.argtypes = [vp]
        L.orc_scene_nodes.argtypes = [vp]
        L.orc_scene_nodes.restype = C.c_int64
        L.orc_closest_hit_batch.argtypes = [vp, C.c_int64, f64, f64, f64, C.c_int, i64, f64, f64]
        L.orc_gbuffer.argtypes = [vp, f32, C.c_int, C.c_int, C.c_float, f32, f32, i64]
        L.orc_ray.argtypes = [C.c_int, f32, f32, C.c_uint32, C.c_float, f32, C.c_uint64,
                              C.c_uint32, f64]
        L.orc_trace.argtypes = [vp, C.c_int, C.c_int, C.c_int, f32, f32, C.c_float, f32,
                                C.c_uint64, C.c_uint32, C.c_int, C.c_int, C.c_int, C.c_int,
                                f64, f64]
        L.orc_reuse.argtypes = [vp, C.c_int, C.c_int, C.c_int, f32, f32, f64, C.c_int, C.c_int,
                                C.c_int, i32, C.c_int, C.c_uint64, C.c_uint32, C.c_int,
                                C.c_float, f32, C.c_int, C.c_int, C.c_int, C.c_int, f64, f64]
        L.orc_reuse_light.argtypes = [vp, C.c_int, C.c_int, f32, C.c_int, C.c_int, C.c_int, i32,
                                      C.c_int, C.c_uint64, f32, C.c_uint64, C.c_uint32, C.c_int,
                                      C.c_int, C.c_int, C.c_int, f64, f64]
        L.orc_mis_weights.argtypes = [vp, C.c_int, C.c_int, C.c_int, f32, f32, f64, C.c_int,
                                      C.c_int, C.c_int, i32, C.c_int, C.c_uint64, C.c_uint32,
                                      C.c_int, C.c_float, f32, C.c_int, C.c_int, i64, f64]
        L.orc_mis_weights.restype = C.c_int
        L.orc_accumulate.argtypes = [vp, C.c_int, C.c_int, C.c_int, f32, f32, C.c_int, C.c_int,
                                     C.c_int, i32, C.c_int, C.c_uint64, C.c_int, C.c_float, f32,
                                     C.c_uint64, C.c_uint32, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.c_int, f64, f64]
        L.orc_random_offsets.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, i32]
        L.orc_random_offsets.restype = C.c_int
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        L.orc_density.argtypes = [C.c_int, f64, f64, f64, f64, C.c_float, f32]
        L.orc_density.restype = C.c_double
        _lib = L
        return L


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (OpenMP)."""
    lib().orc_set_num_threads(int(n))


# ------------------------------------------------------------------------------------
# RNG
# ------------------------------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(np.ascontiguousarray(ctr, dtype=np.uint32),
                            np.ascontiguousarray(key, dtype=np.uint32), out)
    return out


def uniform_pair(seed: int, pix: int, sample: int, stream: int) -> np.ndarray:
    out = np.zeros(2, dtype=np.float64)
    lib().orc_uniform_pair(seed, pix, sample, stream, out)
    return out


# ------------------------------------------------------------------------------------
# Scene
# ------------------------------------------------------------------------------------

class OracleScene:
    """Triangles widened to FP64 plus the oracle's own median-split BVH."""

    def __init__(self, tris: np.ndarray):
        self.tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 3, 3)
        self.handle = lib().orc_scene_create(self.tris.reshape(-1), self.tris.shape[0])

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.orc_scene_destroy(h)
            self.handle = None

    @property
    def num_nodes(self) -> int:
        return int(lib().orc_scene_nodes(self.handle))

    def closest_hit(self, o, d, tmax, brute: bool = False):
        o = np.ascontiguousarray(o, dtype=np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
        n = o.shape[0]
        tm = np.ascontiguousarray(np.broadcast_to(np.asarray(tmax, dtype=np.float64), (n,)))
        tri = np.zeros(n, dtype=np.int64)
        t = np.zeros(n, dtype=np.float64)
        m = np.zeros(n, dtype=np.float64)
        lib().orc_closest_hit_batch(self.handle, n, o, d, tm, int(brute), tri, t, m)
        return tri, t, m


def gbuffer(scene: OracleScene, camera: np.ndarray, W: int, H: int, eps: float):
    """Pinhole primary rays -> float32 pos4/nrm4 [H, W, 4] and hit triangle ids [H, W]."""
    pos = np.zeros((H, W, 4), dtype=np.float32)
    nrm = np.zeros((H, W, 4), dtype=np.float32)
    tri = np.zeros((H, W), dtype=np.int64)
    lib().orc_gbuffer(scene.handle, np.ascontiguousarray(camera, dtype=np.float32), W, H,
                      float(eps), pos, nrm, tri)
    return pos, nrm, tri


def _light(light):
    if light is None:
        return np.zeros(9, dtype=np.float32)
    return np.ascontiguousarray(light, dtype=np.float32).reshape(9)


def ray(effect: int, pos4, nrm4, pix: int, radius: float, light, seed: int, sample: int):
    """Direction and tmax of pixel ``pix``'s step-1 ray (pos4/nrm4: that pixel's 4 floats)."""
    out = np.zeros(4, dtype=np.float64)
    lib().orc_ray(effect, np.ascontiguousarray(pos4, dtype=np.float32),
                  np.ascontiguousarray(nrm4, dtype=np.float32), pix, radius, _light(light), seed,
                  sample, out)
    return out[:3], out[3]


def trace(scene: OracleScene, effect: int, pos4: np.ndarray, nrm4: np.ndarray, radius: float = 0.0,
          light=None, seed: int = 0, sample: int = 0, region=None, out=None):
    """Step 1 of Alg. 1/2 for every pixel of ``region`` (x0, y0, w, h; default: all).

    Returns records float64 [H, W, 8] (z.xyz, n_z.xyz, t, tri; tri = -1 for none) and
    per-pixel margins [H, W]; pixels outside the region hold tri = -1 and margin inf.
    ``out`` = (rec, margin) reuses caller buffers (pixels outside the region untouched).
    """
    H, W = pos4.shape[:2]
    x0, y0, w, h = region if region is not None else (0, 0, W, H)
    if out is not None:
        rec, mg = out
    else:
        rec = np.zeros((H, W, 8), dtype=np.float64)
        rec[..., 7] = -1.0
        mg = np.full((H, W), np.inf)
    lib().orc_trace(scene.handle, effect, W, H, np.ascontiguousarray(pos4, dtype=np.float32),
                    np.ascontiguousarray(nrm4, dtype=np.float32), radius, _light(light), seed,
                    sample, x0, y0, w, h, rec, mg)
    return rec, mg


def _pattern(pattern):
    """(kind, gw, gh, flat offsets, n_offsets, pattern seed).  ``pattern`` = (kind, gw, gh,
    offsets) for groups, boxes and shared offsets, or (PAT_RANDOM, radius_px, n_offsets,
    seed) for per-receiver random offsets in a disk."""
    kind, gw, gh, off = pattern
    if kind == PAT_RANDOM:
        return kind, int(gw), 0, np.zeros(0, dtype=np.int32), int(gh), int(off)
    off = np.zeros((0, 2), dtype=np.int32) if off is None else np.asarray(off, dtype=np.int32)
    return kind, gw, gh, np.ascontiguousarray(off.reshape(-1)), off.shape[0], 0


def random_offsets(seed: int, pix: int, sample: int, radius: int, n_offsets: int) -> np.ndarray:
    """Per-receiver random offsets (pattern kind PAT_RANDOM) of pixel ``pix``: [n, 2] int32."""
    out = np.zeros(2 * 64, dtype=np.int32)
    n = lib().orc_random_offsets(seed, pix, sample, radius, n_offsets, out)
    return out[:2 * n].reshape(n, 2).copy()


def reuse(scene, effect: int, pos4, nrm4, rec, pattern, estimator: int, radius: float = 0.0,
          light=None, region=None, out=None, sample: int = 0):
    """Estimator of Eqs. 17/18/23/24 (or a baseline) for every pixel of ``region``.

    ``pattern`` = (kind, gw, gh, offsets): kind 0 group blocks, 1 centred box,
    2 receiver plus shared offsets [n, 2]; or (3, radius_px, n_offsets, seed): per-receiver
    random offsets drawn for ``sample`` (the records' sample index).  ``scene`` is needed
    only for the unbiased estimator.  Returns (out float64 [H, W], margin [H, W]); ``out``
    = (values, margins) reuses caller buffers.
    """
    H, W = pos4.shape[:2]
    x0, y0, w, h = region if region is not None else (0, 0, W, H)
    kind, gw, gh, off, n_off, pseed = _pattern(pattern)
    if out is not None:
        out, mg = out
    else:
        out = np.full((H, W), np.nan)
        mg = np.full((H, W), np.inf)
    lib().orc_reuse(scene.handle if scene is not None else None, effect, W, H,
                    np.ascontiguousarray(pos4, dtype=np.float32),
                    np.ascontiguousarray(nrm4, dtype=np.float32),
                    np.ascontiguousarray(rec, dtype=np.float64), kind, gw, gh, off, n_off, pseed,
                    sample, estimator, radius, _light(light), x0, y0, w, h, out, mg)
    return out, mg


def reuse_light(scene, pos4, pattern, light, seed: int, sample: int, region=None, out=None):
    """Unbiased light-sample reuse for shadows (Light(N U)): the mean visibility of the
    segments from each receiver to its members' light samples (sample `sample`, key
    `seed`).  Returns (out float64 [H, W], margin [H, W])."""
    H, W = pos4.shape[:2]
    x0, y0, w, h = region if region is not None else (0, 0, W, H)
    kind, gw, gh, off, n_off, pseed = _pattern(pattern)
    if out is not None:
        out, mg = out
    else:
        out = np.full((H, W), np.nan)
        mg = np.full((H, W), np.inf)
    lib().orc_reuse_light(scene.handle, W, H, np.ascontiguousarray(pos4, dtype=np.float32), kind,
                          gw, gh, off, n_off, pseed, _light(light), seed, sample, x0, y0, w, h,
                          out, mg)
    return out, mg


def density(effect: int, z, nz, x, nx, radius: float = 0.0, light=None) -> float:
    """Biased density p~(z | x) of Eq. 15 (AO) or Eq. 21 (shadow)."""
    a = [np.ascontiguousarray(v, dtype=np.float64).reshape(3) for v in (z, nz, x, nx)]
    return float(lib().orc_density(effect, *a, radius, _light(light)))


def mis_weights(scene, effect: int, pos4, nrm4, rec, pattern, estimator: int, px: int, py: int,
                radius: float = 0.0, light=None, sample: int = 0):
    """(member pixel ids, weight matrix w[j][k]) seen by receiver (px, py)."""
    H, W = pos4.shape[:2]
    kind, gw, gh, off, n_off, pseed = _pattern(pattern)
    mem = np.zeros(64, dtype=np.int64)
    w = np.zeros(64 * 64, dtype=np.float64)
    n = lib().orc_mis_weights(scene.handle if scene is not None else None, effect, W, H,
                              np.ascontiguousarray(pos4, dtype=np.float32),
                              np.ascontiguousarray(nrm4, dtype=np.float32),
                              np.ascontiguousarray(rec, dtype=np.float64), kind, gw, gh, off,
                              n_off, pseed, sample, estimator, radius, _light(light), px, py, mem,
                              w)
    return mem[:n].copy(), w[:n * n].reshape(n, n).copy()


def accumulate(scene, effect: int, pos4, nrm4, pattern, estimator: int, radius: float = 0.0,
               light=None, seed: int = 0, sample0: int = 0, M: int = 1, region=None):
    """Per-pixel mean and variance of the per-sample estimate over samples
    sample0 .. sample0 + M - 1, for the pixels of ``region`` -> ([h, w], [h, w])."""
    H, W = pos4.shape[:2]
    x0, y0, w, h = region if region is not None else (0, 0, W, H)
    kind, gw, gh, off, n_off, pseed = _pattern(pattern)
    mean = np.zeros(w * h, dtype=np.float64)
    var = np.zeros(w * h, dtype=np.float64)
    lib().orc_accumulate(scene.handle, effect, W, H, np.ascontiguousarray(pos4, dtype=np.float32),
                         np.ascontiguousarray(nrm4, dtype=np.float32), kind, gw, gh, off, n_off,
                         pseed, estimator, radius, _light(light), seed, sample0, M, x0, y0, w, h,
                         mean, var)
    return mean.reshape(h, w), var.reshape(h, w)
