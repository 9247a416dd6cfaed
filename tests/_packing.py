"""NumPy reference of the packed storage formats (test infrastructure).

Packs oracle-made inputs the way include/occ.h describes the PACKED formats, so the CUDA
path can be fed packed data that it did not produce, and unpacks them again for the
oracle.  Octahedral normals: Cigolle et al., JCGT 2014 (2 x 16-bit snorm); occluder
points as offsets from the source receiver, three 19-bit mantissas with a shared exponent.
"""
import numpy as np

OCT_INVALID = np.uint32(0x80008000)


def oct_encode(n: np.ndarray) -> np.ndarray:
    """Unit vectors [..., 3] -> uint32 codes, computed in FP32 step by step."""
    n = np.asarray(n, dtype=np.float32)
    x, y, z = n[..., 0], n[..., 1], n[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):   # zero vectors of empty records
        inv = np.float32(1.0) / ((np.abs(x) + np.abs(y)) + np.abs(z))
        px, py = x * inv, y * inv
    sx = np.where(px >= 0, np.float32(1), np.float32(-1))
    sy = np.where(py >= 0, np.float32(1), np.float32(-1))
    fx = (np.float32(1) - np.abs(py)) * sx
    fy = (np.float32(1) - np.abs(px)) * sy
    lower = z < 0
    px, py = np.where(lower, fx, px), np.where(lower, fy, py)
    with np.errstate(invalid="ignore"):
        qx = np.rint(np.nan_to_num(np.clip(px, -1, 1)) * np.float32(32767)).astype(np.int32)
        qy = np.rint(np.nan_to_num(np.clip(py, -1, 1)) * np.float32(32767)).astype(np.int32)
    return ((qx & 0xFFFF) | ((qy & 0xFFFF) << 16)).astype(np.uint32)


def oct_decode(c: np.ndarray) -> np.ndarray:
    """uint32 codes -> unit vectors [..., 3] in FP64.  The unfolded vector is formed in
    integers (units of 1/32767), so z and the fold decision are exact."""
    c = np.asarray(c, dtype=np.uint32)
    qx = (c & 0xFFFF).astype(np.uint16).view(np.int16).astype(np.int64)
    qy = (c >> 16).astype(np.uint16).view(np.int16).astype(np.int64)
    qz = 32767 - np.abs(qx) - np.abs(qy)
    lower = qz < 0
    tx = qx.copy()
    qx = np.where(lower, (32767 - np.abs(qy)) * np.where(tx >= 0, 1, -1), qx)
    qy = np.where(lower, (32767 - np.abs(tx)) * np.where(qy >= 0, 1, -1), qy)
    v = np.stack([qx, qy, qz], axis=-1).astype(np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        return v / np.linalg.norm(v, axis=-1, keepdims=True)


def pack_gbuffer(pos4: np.ndarray, nrm4: np.ndarray) -> np.ndarray:
    """FP32 G-buffer -> packed plane [H, W, 4] float32 (x.xyz, code bits)."""
    out = np.zeros(pos4.shape, dtype=np.float32)
    out[..., :3] = pos4[..., :3]
    code = oct_encode(nrm4[..., :3])
    code = np.where(pos4[..., 3] != 0, code, OCT_INVALID).astype(np.uint32)
    out[..., 3] = code.view(np.float32)
    return out


def unpack_gbuffer(packed: np.ndarray):
    """Packed plane -> (pos4, nrm4) float32 with the decoded normals (for the oracle)."""
    code = packed[..., 3].copy().view(np.uint32)
    valid = code != OCT_INVALID
    pos = np.zeros(packed.shape, dtype=np.float32)
    nrm = np.zeros(packed.shape, dtype=np.float32)
    pos[..., :3] = packed[..., :3]
    pos[..., 3] = valid.astype(np.float32)
    n = oct_decode(code)
    nrm[..., :3] = np.where(valid[..., None], n, 0.0).astype(np.float32)
    return pos, nrm


MANT_MAX = (1 << 18) - 1
EXP_BIAS = 60


def _offset_exponent(d: np.ndarray) -> np.ndarray:
    """E = floor(log2 max|d_i|) + 43, clamped to 0..63 (0 for a zero offset)."""
    M = np.abs(d).max(axis=-1)
    with np.errstate(divide="ignore"):
        _, e = np.frexp(M)                     # M = f 2^e, f in [0.5, 1): floor(log2 M) = e - 1
    return np.where(M > 0, np.clip(e - 1 + 43, 0, 63), 0).astype(np.int64)


def pack_records(orec: np.ndarray, pos4: np.ndarray) -> np.ndarray:
    """Oracle records [H, W, 8] -> packed plane [H, W, 4] float32 (16-byte records):
    d = z - x in FP64, shared exponent, mantissas rounded to nearest even."""
    H, W = orec.shape[:2]
    hit = orec[..., 7] >= 0
    off = orec[..., :3] - pos4[..., :3].astype(np.float64)
    E = _offset_exponent(off)
    m = np.clip(np.rint(off * np.exp2(EXP_BIAS - E)[..., None]), -MANT_MAX, MANT_MAX)
    m = (m.astype(np.int64) & 0x7FFFF).astype(np.uint64)
    w64 = (m[..., 0] | (m[..., 1] << np.uint64(19)) | (m[..., 2] << np.uint64(38))
           | (E.astype(np.uint64) << np.uint64(57)) | np.uint64(1 << 63))
    words = np.zeros((H, W, 4), dtype=np.uint32)
    words[..., 0] = (w64 & 0xFFFFFFFF).astype(np.uint32)
    words[..., 1] = (w64 >> np.uint64(32)).astype(np.uint32)
    words[..., 2] = oct_encode(orec[..., 3:6])
    words[..., 3] = orec[..., 7].astype(np.int32).view(np.uint32)
    words[~hit] = 0
    words[~hit, 3] = np.uint32(0xFFFFFFFF)
    return words.view(np.float32)


def fma_f32(a: np.ndarray, x: np.ndarray) -> np.ndarray:
    """fl32(a + x) of the exact real sum, for FP64 a and FP32-valued x (as an FMA with an
    exact product a rounds it): TwoSum gives the exact sum as s + e in FP64; rounding s to
    FP32 matches rounding s + e except when s lies exactly halfway between two FP32
    values and e != 0, where e decides."""
    s = a + x
    bb = s - x
    e = (x - (s - bb)) + (a - bb)
    r = s.astype(np.float32)
    r64 = r.astype(np.float64)
    up = np.nextafter(r, np.float32(np.inf))
    dn = np.nextafter(r, np.float32(-np.inf))
    lo = np.where(r64 <= s, r, dn)
    hi = np.where(r64 <= s, up, r)
    mid = (s - lo.astype(np.float64)) == (hi.astype(np.float64) - s)
    return np.where(mid & (e > 0), hi, np.where(mid & (e < 0), lo, r))


def unpack_records(packed: np.ndarray, pos4: np.ndarray) -> np.ndarray:
    """Packed plane -> the oracle's FP64 record layout, z rebuilt as the format defines it:
    fmaf(m, 2^(E - 60), x) in FP32 (the product is exact, so this is one rounding of the
    exact sum)."""
    w = packed.view(np.uint32)
    H, W = packed.shape[:2]
    rec = np.zeros((H, W, 8))
    tri = w[..., 3].view(np.int32)
    hit = tri >= 0
    w64 = w[..., 0].astype(np.uint64) | (w[..., 1].astype(np.uint64) << np.uint64(32))
    E = ((w64 >> np.uint64(57)) & np.uint64(63)).astype(np.int64)
    unit = np.exp2(E - EXP_BIAS)
    comps = []
    for k in range(3):
        v = ((w64 >> np.uint64(19 * k)) & np.uint64(0x7FFFF)).astype(np.int64)
        v = np.where(v >= (1 << 18), v - (1 << 19), v)
        comps.append(v.astype(np.float64) * unit)
    a = np.stack(comps, axis=-1)
    x = pos4[..., :3].astype(np.float32).astype(np.float64)
    z = fma_f32(a, x).astype(np.float64)
    n = oct_decode(w[..., 2])
    rec[..., :3] = np.where(hit[..., None], z, 0.0)
    rec[..., 3:6] = np.where(hit[..., None], n, 0.0)
    rec[..., 7] = np.where(hit, tri, -1)
    return rec
