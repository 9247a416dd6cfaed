"""The NumPy reference codec of the packed formats (no GPU): the FP32 fused multiply-add
emulation against exact rational rounding, the offset round trip bound, octahedral normals."""
from fractions import Fraction

import numpy as np

from tests import _packing as PK


def _rn32(fr: Fraction) -> np.float32:
    f = np.float32(float(fr))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    return min(cands, key=lambda c: (abs(Fraction(float(c)) - fr),
                                     int(np.float32(c).view(np.uint32)) & 1))


def test_fma_emulation_rounds_the_exact_sum():
    rng = np.random.default_rng(1)
    n = 3000
    x = rng.uniform(-32, 32, n).astype(np.float32).astype(np.float64)
    a = rng.integers(-2**18, 2**18, n) * np.exp2(rng.integers(-60, 3, n))
    k = n // 2                                   # halfway cases, nudged by 2^-60 either way
    ulp = np.spacing(np.abs(x[:k].astype(np.float32))).astype(np.float64)
    a[:k] = ulp / 2 * np.sign(rng.normal(size=k)) + rng.choice([0, 1, -1], k) * 2.0 ** -60
    got = PK.fma_f32(a, x)
    want = np.array([_rn32(Fraction(float(a[i])) + Fraction(float(x[i]))) for i in range(n)])
    assert np.array_equal(got, want)


def test_offset_round_trip_bound():
    rng = np.random.default_rng(2)
    H, W = 48, 40
    pos = np.zeros((H, W, 4), np.float32)
    pos[..., :3] = rng.uniform(-16, 16, (H, W, 3)).astype(np.float32)
    pos[..., 3] = 1
    d = rng.normal(size=(H, W, 3)) * 10 ** rng.uniform(-6, 1.3, (H, W, 1))
    orec = np.zeros((H, W, 8))
    orec[..., :3] = pos[..., :3].astype(np.float64) + d
    n = rng.normal(size=(H, W, 3))
    orec[..., 3:6] = n / np.linalg.norm(n, axis=-1, keepdims=True)
    orec[..., 7] = np.arange(H * W).reshape(H, W)
    orec[3, 5, 7] = -1
    u = PK.unpack_records(PK.pack_records(orec, pos), pos)
    hit = orec[..., 7] >= 0
    err = np.abs(u[..., :3] - orec[..., :3]).max(-1)[hit]
    dmax = np.abs(d).max(-1)[hit]
    ulp = np.spacing(np.abs(orec[..., :3]).astype(np.float32)).max(-1)[hit]
    assert np.all(err <= 2.0 ** -18 * dmax + ulp)
    assert np.array_equal(u[..., 7], np.where(hit, orec[..., 7], -1))
    assert np.all(u[~hit, :6] == 0)
    assert np.abs(u[..., 3:6][hit] - orec[..., 3:6][hit]).max() < 2e-4   # octahedral 2 x 16 bit


def test_octahedral_codes_are_exact_on_the_axes_and_unit_length():
    axes = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    assert np.array_equal(PK.oct_decode(PK.oct_encode(axes)), axes)
    rng = np.random.default_rng(3)
    v = rng.normal(size=(5000, 3))
    v /= np.linalg.norm(v, axis=-1, keepdims=True)
    w = PK.oct_decode(PK.oct_encode(v))
    assert np.allclose(np.linalg.norm(w, axis=-1), 1.0, atol=1e-12)
    assert np.abs(w - v).max() < 2e-4
