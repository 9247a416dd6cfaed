"""NumPy reference of the packed storage formats (test infrastructure).

Packs oracle-made inputs the way include/occ.h describes the PACKED formats, so the CUDA
path can be fed packed data that it did not produce, and unpacks them again for the
oracle.  Octahedral normals: Cigolle et al., JCGT 2014 (2 x 16-bit snorm); occluder
points as 21-bit fixed-point offsets from the source receiver (unit scale * 2^-20).
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


def pack_records(orec: np.ndarray, pos4: np.ndarray, scale: float) -> np.ndarray:
    """Oracle records [H, W, 8] -> packed plane [H, W, 4] float32 (16-byte records)."""
    H, W = orec.shape[:2]
    hit = orec[..., 7] >= 0
    off = orec[..., :3] - pos4[..., :3].astype(np.float64)
    q = np.clip(np.rint(off * (2.0 ** 20 / np.float64(np.float32(scale)))), -1048575, 1048575)
    q = (q.astype(np.int64) & 0x1FFFFF).astype(np.uint64)
    w64 = (q[..., 0] | (q[..., 1] << np.uint64(21)) | (q[..., 2] << np.uint64(42))
           | np.uint64(1 << 63))
    words = np.zeros((H, W, 4), dtype=np.uint32)
    words[..., 0] = (w64 & 0xFFFFFFFF).astype(np.uint32)
    words[..., 1] = (w64 >> np.uint64(32)).astype(np.uint32)
    words[..., 2] = oct_encode(orec[..., 3:6])
    words[..., 3] = orec[..., 7].astype(np.int32).view(np.uint32)
    words[~hit] = 0
    words[~hit, 3] = np.uint32(0xFFFFFFFF)
    return words.view(np.float32)


def unpack_records(packed: np.ndarray, pos4: np.ndarray, scale: float) -> np.ndarray:
    """Packed plane -> the oracle's FP64 record layout (z rebuilt from the offsets)."""
    w = packed.view(np.uint32)
    H, W = packed.shape[:2]
    rec = np.zeros((H, W, 8))
    tri = w[..., 3].view(np.int32)
    hit = tri >= 0
    w64 = w[..., 0].astype(np.uint64) | (w[..., 1].astype(np.uint64) << np.uint64(32))
    unit = np.float64(np.float32(np.float32(scale) * np.float32(1.0 / 1048576.0)))
    comps = []
    for k in range(3):
        v = ((w64 >> np.uint64(21 * k)) & np.uint64(0x1FFFFF)).astype(np.int64)
        v = np.where(v >= (1 << 20), v - (1 << 21), v)
        comps.append(v.astype(np.float64) * unit)
    x = pos4[..., :3].astype(np.float64)
    z = x + np.stack(comps, axis=-1)
    n = oct_decode(w[..., 2])
    rec[..., :3] = np.where(hit[..., None], z, 0.0)
    rec[..., 3:6] = np.where(hit[..., None], n, 0.0)
    rec[..., 7] = np.where(hit, tri, -1)
    return rec
