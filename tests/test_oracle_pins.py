"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
implementation of the same published generator, closed-form moments and
integrals, analytic intersections, brute force, invariants of the balance
heuristic (Eq. 11), the special cases Sec. 4 implies (no occluder, K = 1,
fully lit or blocked lights, the guard), and convergence of the unbiased
estimators (Eqs. 17, 23) to a high-spp no-reuse reference (Sec. 6, App. J/K).
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

AO, SH = 0, 1
NOREUSE, BIASED, UNBIASED, BOXMEAN = 0, 1, 2, 3
GROUP, BOX, OFFS, RAND = 0, 1, 2, 3


# --------------------------------------------------------------------------------------
# Philox4x32-10: oracle vs Triton's implementation of the same published generator
# --------------------------------------------------------------------------------------

def test_philox_matches_triton_reference(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(123)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64)
    key = rng.integers(0, 2**32, size=(64, 2), dtype=np.uint64)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 2**32 - 1
    key[1] = 2**32 - 1
    req = json.dumps({"ctr": ctr.astype(np.int64).tolist(), "key": key.astype(np.int64).tolist()})
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_triton_philox.py")],
                         input=req, capture_output=True, text=True, env=env, timeout=600)
    if res.returncode != 0:
        pytest.skip("Triton interpreter unavailable: " + res.stderr[-300:])
    ref = np.array(json.loads(res.stdout), dtype=np.uint64)
    got = np.array([orc.philox4x32_10(c, k) for c, k in zip(ctr, key)], dtype=np.uint64)
    assert np.array_equal(got, ref)


def test_uniforms_are_24bit_and_uniform(orc):
    n = 20000
    u = np.array([orc.uniform_pair(99, p, 3, 0) for p in range(n)])
    assert np.all(u >= 0.0) and np.all(u < 1.0)
    assert np.all(u * 2**24 == np.floor(u * 2**24))
    for c in range(2):
        hist, _ = np.histogram(u[:, c], bins=20, range=(0, 1))
        chi2 = ((hist - n / 20) ** 2 / (n / 20)).sum()
        assert chi2 < 45.3  # 19 dof, p = 0.001
    # different streams / samples give different words
    assert not np.array_equal(orc.uniform_pair(99, 5, 3, 0), orc.uniform_pair(99, 5, 3, 1))
    assert not np.array_equal(orc.uniform_pair(99, 5, 3, 0), orc.uniform_pair(99, 5, 4, 0))


# --------------------------------------------------------------------------------------
# Eq. 2: cosine-weighted hemisphere directions
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("normal", [(0, 0, 1), (0, 0, -1), (1, 0, 0), (0.3, -0.5, 0.81),
                                    (-0.6, 0.0, -0.8)])
def test_cosine_direction_moments(orc, normal):
    n = np.array(normal, dtype=np.float64)
    n = (n / np.linalg.norm(n)).astype(np.float32)
    pos = np.array([0.5, -1.0, 2.0, 1.0], dtype=np.float32)
    nrm = np.array([n[0], n[1], n[2], 0.0], dtype=np.float32)
    N = 40000
    dirs = np.array([orc.ray(AO, pos, nrm, p, 0.7, None, 11, 0)[0] for p in range(N)])
    tmax = orc.ray(AO, pos, nrm, 0, 0.7, None, 11, 0)[1]
    assert tmax == pytest.approx(0.7, rel=1e-7)
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-6)
    c = dirs @ n.astype(np.float64)
    assert c.min() >= -1e-7
    # p(w) = cos/pi  =>  E[cos] = 2/3, E[cos^2] = 1/2, Var[cos] = 1/18
    sig = math.sqrt((1 / 2 - 4 / 9) / N)
    assert abs(c.mean() - 2 / 3) < 4 * sig
    sig2 = math.sqrt((1 / 3 - 1 / 4) / N)  # Var[cos^2] = E[cos^4] - 1/4 = 1/3 - 1/4
    assert abs((c ** 2).mean() - 0.5) < 4 * sig2
    # azimuth is uniform: the tangential part has zero mean in every direction
    tang = dirs - np.outer(c, n)
    assert np.all(np.abs(tang.mean(axis=0)) < 4 * math.sqrt(0.5 / N))


def test_shadow_sample_uniform_on_light(orc):
    light = synth.light_c3().as_array()
    pos = np.array([0.2, 0.1, 0.0, 1.0], dtype=np.float32)
    nrm = np.array([0, 0, 1, 0], dtype=np.float32)
    N = 20000
    ys = []
    for p in range(N):
        d, tmax = orc.ray(SH, pos, nrm, p, 0.0, light, 5, 0)
        ys.append(pos[:3].astype(np.float64) + d * tmax)
    ys = np.array(ys)
    c, eu, ev = light[:3], light[3:6], light[6:9]
    assert np.allclose(ys[:, 2], 4.0, atol=1e-9)
    a = (ys - c) @ eu / (eu @ eu)
    b = (ys - c) @ ev / (ev @ ev)
    assert a.min() >= -0.5 and a.max() < 0.5 and b.min() >= -0.5 and b.max() < 0.5
    for v in (a, b):
        hist, _ = np.histogram(v, bins=10, range=(-0.5, 0.5))
        assert ((hist - N / 10) ** 2 / (N / 10)).sum() < 27.9  # 9 dof, p = 0.001


# --------------------------------------------------------------------------------------
# Closest hit: analytic cases, watertightness, BVH == brute force, tie rule
# --------------------------------------------------------------------------------------

def _scene(tris):
    import oracle
    return oracle.OracleScene(np.asarray(tris, dtype=np.float32))


def test_closest_hit_analytic(orc):
    sc = _scene([[[0, 0, 1], [1, 0, 1], [0, 1, 1]]])
    o = [[0.2, 0.2, 0.0], [0.2, 0.2, 0.0], [0.6, 0.6, 0.0], [0.2, 0.2, 0.0], [0.2, 0.2, 2.0],
         [0.2, 0.2, 0.0], [0.2, 0.2, 0.0]]
    d = [[0, 0, 1], [0, 0, 2], [0, 0, 1], [0, 0, -1], [0, 0, -1], [0, 0, 1], [0, 0, 1]]
    tmax = [10, 10, 10, 10, 10, 1.0, 0.999]
    tri, t, _ = sc.closest_hit(o, d, tmax)
    assert tri.tolist() == [0, 0, -1, -1, 0, 0, -1]
    assert t[0] == 1.0 and t[1] == 0.5 and t[4] == 1.0 and t[5] == 1.0


def test_tie_rule_prefers_smaller_t_then_smaller_id(orc):
    tri_a = [[0, 0, 1], [1, 0, 1], [0, 1, 1]]
    tri_b = [[0, 0, 2], [1, 0, 2], [0, 1, 2]]
    sc = _scene([tri_b, tri_a, tri_a])   # ids: 0 at z=2, 1 and 2 coincide at z=1
    tri, t, m = sc.closest_hit([[0.2, 0.2, 0]], [[0, 0, 1]], [10])
    assert tri[0] == 1 and t[0] == 1.0
    assert m[0] == 0.0   # two triangles at the same t: flagged as ambiguous


def test_watertight_fan(orc):
    k = 12
    ang = np.arange(k) * 2 * np.pi / k
    rim = np.stack([np.cos(ang), np.sin(ang), np.ones(k)], axis=1)
    ctr = np.array([0.0, 0.0, 1.0])
    tris = [[ctr, rim[i], rim[(i + 1) % k]] for i in range(k)]
    sc = _scene(tris)
    # rays through the shared edges and the shared vertex, and random rays in the disk
    pts = [np.zeros(2)] + [0.5 * np.array([math.cos(a), math.sin(a)]) for a in ang]
    rng = np.random.default_rng(5)
    pts += list(rng.uniform(-0.6, 0.6, size=(500, 2)))
    o = np.array([[p[0], p[1], 0.0] for p in pts])
    d = np.tile([0.0, 0.0, 1.0], (len(pts), 1))
    tri, t, _ = sc.closest_hit(o, d, 10.0)
    assert np.all(tri >= 0)
    assert np.allclose(t, 1.0)
    # oblique rays through the vertex from many directions
    dirs = rng.normal(size=(300, 3))
    dirs[:, 2] = np.abs(dirs[:, 2]) + 0.2
    o2 = ctr[None, :] - dirs
    tri2, t2, _ = sc.closest_hit(o2, dirs, 10.0)
    assert np.all(tri2 >= 0)
    assert np.allclose(t2, 1.0, rtol=1e-12)


@pytest.mark.parametrize("which", ["c1", "terrain"])
def test_bvh_equals_brute_force(orc, which):
    if which == "c1":
        scene = synth.scene_c1()
    else:
        scene = synth.scene_terrain(grid=48, n_spheres=6, n_boxes=60, seed=4, sphere_subdiv=2)
    sc = orc.OracleScene(scene.tris)
    v = scene.tris.reshape(-1, 3)
    lo, hi = v.min(0), v.max(0)
    rng = np.random.default_rng(17)
    n = 4000
    o = rng.uniform(lo, hi, size=(n, 3))
    d = rng.normal(size=(n, 3))
    tmax = rng.uniform(0.1, 20.0, size=n)
    a = sc.closest_hit(o, d, tmax, brute=False)
    b = sc.closest_hit(o, d, tmax, brute=True)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert (a[0] >= 0).mean() > 0.2


def test_gbuffer_plane_analytic(orc):
    scene = synth.scene_plane_only()
    sc = orc.OracleScene(scene.tris)
    cam = synth.Camera(eye=(0.3, -5.0, 3.0), target=(0.0, 0.0, 0.0), vfov_deg=60.0)
    W, H = 24, 16
    pos, nrm, tri = orc.gbuffer(sc, cam.as_array(), W, H, scene.eps)
    eye = np.array(cam.eye)
    valid = pos[..., 3] > 0
    assert valid.mean() > 0.5
    # every valid receiver lies eps above the plane z = 0 with normal +z (faces the camera)
    assert np.allclose(pos[valid][:, 2], scene.eps, rtol=1e-6)
    assert np.allclose(nrm[valid][:, :3], [0, 0, 1])
    # the receiver lies on the primary ray: (p - eps n) - eye is parallel to the pixel ray
    f = -eye / np.linalg.norm(eye)
    rt = np.cross(f, [0, 0, 1.0])
    rt /= np.linalg.norm(rt)
    up = np.cross(rt, f)
    th = math.tan(math.radians(30.0))
    for py, px in np.argwhere(valid)[::7]:
        sx = (2 * (px + 0.5) / W - 1) * th * W / H
        sy = (1 - 2 * (py + 0.5) / H) * th
        dd = f + sx * rt + sy * up
        t = -eye[2] / dd[2]
        assert np.allclose(pos[py, px, :3] - [0, 0, scene.eps], eye + t * dd, atol=1e-5)


# --------------------------------------------------------------------------------------
# Densities: the oracle's simplified forms vs Eqs. 13-15 and 20-21 written out
# --------------------------------------------------------------------------------------

def _unit(v):
    return v / np.linalg.norm(v)


def test_ao_density_matches_eqs_13_15(orc):
    rng = np.random.default_rng(2)
    R = 0.8
    hits = 0
    for _ in range(2000):
        x = rng.normal(size=3)
        nx = _unit(rng.normal(size=3))
        z = x + rng.normal(size=3) * 0.4
        nz = _unit(rng.normal(size=3))
        got = orc.density(AO, z, nz, x, nx, radius=R)
        r = np.linalg.norm(x - z)
        w_xz = (z - x) / r
        w_zx = (x - z) / r
        cos_x = max(0.0, nx @ w_xz)
        J = max(0.0, nz @ w_zx) / r ** 2                      # Eq. 13
        want = cos_x * J / math.pi * (r <= np.float32(R))     # Eq. 15 without Occ
        assert got == pytest.approx(want, rel=1e-12, abs=1e-300)
        hits += want > 0
    assert hits > 300


def test_shadow_density_matches_eqs_20_21(orc):
    rng = np.random.default_rng(3)
    hits = 0
    for _ in range(3000):
        c = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(3, 5)])
        eu = np.array([rng.uniform(0.5, 2), 0, 0])
        ev = np.array([0, -rng.uniform(0.3, 1.5), 0])
        light = np.concatenate([c, eu, ev]).astype(np.float32)
        c, eu, ev = light[:3].astype(float), light[3:6].astype(float), light[6:].astype(float)
        nL = _unit(np.cross(eu, ev))
        area = np.linalg.norm(np.cross(eu, ev))
        x = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-0.5, 0.5)])
        # aim at a point near the light (about 70 % land inside the rectangle)
        tgt = c + rng.uniform(-0.6, 0.6) * eu + rng.uniform(-0.6, 0.6) * ev
        z = x + rng.uniform(0.05, 1.02) * (tgt - x)
        nz = _unit(rng.normal(size=3))
        got = orc.density(SH, z, nz, x, [0, 0, 1.0], light=light)
        # Eq. 20 with the light point y' where the ray x -> z meets the light plane
        d = z - x
        s = (nL @ (c - x)) / (nL @ d)
        yp = x + s * d
        q = yp - c
        inside = abs(q @ eu / (eu @ eu)) <= 0.5 and abs(q @ ev / (ev @ ev)) <= 0.5
        chi = (nL @ d) < 0 and s > 1 and inside
        cos_z = max(0.0, nz @ _unit(x - z))
        cos_y = max(0.0, nL @ _unit(x - yp))
        if chi and cos_y > 0:
            J = cos_z * np.linalg.norm(x - yp) ** 2 / (cos_y * np.linalg.norm(x - z) ** 2)
            want = J / area                                   # Eq. 21 without Occ
        else:
            want = 0.0
        assert got == pytest.approx(want, rel=1e-11, abs=1e-300)
        hits += want > 0
    assert hits > 600


@pytest.mark.parametrize("h_over_R", [0.25, 0.5, 0.9])
def test_ao_density_integrates_to_occluded_fraction(orc, h_over_R):
    """Integral of p_AO(z|x) over a parallel plane = 1 - AO = 1 - (h/R)^2 (from Eq. 1)."""
    from scipy import integrate
    R = 1.0
    h = h_over_R * R
    x = np.zeros(3)
    nx = np.array([0, 0, 1.0])
    nz = np.array([0, 0, -1.0])

    def f(rho):
        return orc.density(AO, [rho, 0.0, h], nz, x, nx, radius=R) * 2 * math.pi * rho

    rmax = math.sqrt(R * R - h * h)
    val, _ = integrate.quad(f, 0.0, rmax, epsabs=1e-13, epsrel=1e-11, limit=200)
    assert val == pytest.approx(1 - h_over_R ** 2, rel=1e-8)
    assert orc.density(AO, [rmax * 1.001, 0.0, h], nz, x, nx, radius=R) == 0.0


def test_shadow_density_integrates_to_one_under_full_blocker(orc):
    """A blocker plane under the whole light: integral of p_Sh(z|x) over it = 1 (Eq. 19)."""
    from scipy import integrate
    light = np.array([0.3, -0.2, 4.0, 1.0, 0, 0, 0, -0.5, 0], dtype=np.float32)
    c, eu, ev = light[:3].astype(float), light[3:6].astype(float), light[6:].astype(float)
    x = np.array([0.7, 0.4, 0.0])
    hb = 1.5
    lam = hb / c[2]
    # support on the blocker: z = x + lam (y - x), y on the light
    xlo = x[0] + lam * (c[0] - 0.5 * abs(eu[0]) - x[0])
    xhi = x[0] + lam * (c[0] + 0.5 * abs(eu[0]) - x[0])
    ylo = x[1] + lam * (c[1] - 0.5 * abs(ev[1]) - x[1])
    yhi = x[1] + lam * (c[1] + 0.5 * abs(ev[1]) - x[1])
    nz = np.array([0, 0, -1.0])

    def f(yy, xx):
        return orc.density(SH, [xx, yy, hb], nz, x, [0, 0, 1.0], light=light)

    val, _ = integrate.dblquad(f, xlo, xhi, ylo, yhi, epsabs=1e-11, epsrel=1e-9)
    assert val == pytest.approx(1.0, rel=1e-7)
    assert f(0.5 * (ylo + yhi), xhi + 0.01) == 0.0


# --------------------------------------------------------------------------------------
# Whole-estimator special cases
# --------------------------------------------------------------------------------------

PATTERNS = [(GROUP, 2, 2, None), (GROUP, 4, 2, None), (BOX, 3, 3, None),
            (OFFS, 0, 0, synth.disk_offsets(8, 6.0, seed=3)), (RAND, 6, 7, 1234)]


def test_random_offsets_uniform_on_the_disk_lattice(orc):
    """Per-receiver random neighbour sets (the per-receiver form of N_i, Eq. 8): every offset
    is a lattice point of the disk other than (0, 0), a receiver's offsets are distinct, and
    each slot is uniform over the lattice points (chi^2); sets change with the sample and
    the seed, and a seed above 32 bits uses its high word."""
    R = 6
    pts = [(x, y) for y in range(-R, R + 1) for x in range(-R, R + 1)
           if x * x + y * y <= R * R and (x, y) != (0, 0)]
    index = {p: i for i, p in enumerate(pts)}
    n = 12000
    counts = np.zeros((2, len(pts)))
    for p in range(n):
        offs = orc.random_offsets(77, p, p % 5, R, 7)
        assert len(offs) == 7 and len({tuple(o) for o in offs}) == 7
        assert all(tuple(o) in index for o in offs)
        counts[0, index[tuple(offs[0])]] += 1
        counts[1, index[tuple(offs[6])]] += 1
    exp, dof = n / len(pts), len(pts) - 1
    for c in counts:
        assert ((c - exp) ** 2 / exp).sum() < dof + 5 * math.sqrt(2 * dof)
    assert not np.array_equal(orc.random_offsets(77, 5, 0, R, 7), orc.random_offsets(77, 5, 1, R, 7))
    assert not np.array_equal(orc.random_offsets(77, 5, 0, R, 7), orc.random_offsets(78, 5, 0, R, 7))
    assert not np.array_equal(orc.random_offsets(77, 5, 0, R, 7),
                              orc.random_offsets(77 + 2**32, 5, 0, R, 7))
    # a disk of radius 1 has four lattice points besides the origin: four slots take all
    assert sorted(map(tuple, orc.random_offsets(3, 9, 0, 1, 4))) == [(-1, 0), (0, -1), (0, 1), (1, 0)]


def _grid_case(scene, W=24, H=16, spacing=0.05):
    pos, nrm = synth.receiver_grid(W, H, spacing, z=scene.eps)
    return pos, nrm


@pytest.mark.parametrize("pattern", PATTERNS)
def test_ao_unoccluded_plane_is_one(orc, pattern):
    scene = synth.scene_plane_only()
    sc = orc.OracleScene(scene.tris)
    pos, nrm = _grid_case(scene)
    for s in range(3):
        rec, _ = orc.trace(sc, AO, pos, nrm, radius=1.0, seed=4, sample=s)
        assert np.all(rec[..., 7] < 0)
        for est in (NOREUSE, BIASED, UNBIASED, BOXMEAN):
            out, _ = orc.reuse(sc, AO, pos, nrm, rec, pattern, est, radius=1.0)
            assert np.all(out == 1.0)


def _image_mean_over_samples(orc, sc, effect, pos, nrm, pattern, est, M, seed, radius=0.0,
                             light=None):
    means = []
    for s in range(M):
        rec, _ = orc.trace(sc, effect, pos, nrm, radius=radius, light=light, seed=seed, sample=s)
        out, _ = orc.reuse(sc, effect, pos, nrm, rec, pattern, est, radius=radius, light=light,
                           sample=s)
        means.append(out.mean())
    means = np.array(means)
    return means.mean(), means.std(ddof=1) / math.sqrt(M)


@pytest.mark.parametrize("h_over_R", [0.25, 0.5, 0.9])
@pytest.mark.parametrize("pattern", [PATTERNS[1], PATTERNS[2], PATTERNS[3]])
def test_ao_parallel_plane_closed_form(orc, h_over_R, pattern):
    """Eq. 1 under an infinite parallel plane at height h: AO = (h/R)^2."""
    R = 1.0
    scene = synth.scene_parallel_plane(h_over_R * R)
    sc = orc.OracleScene(scene.tris)
    pos, nrm = _grid_case(scene)
    h = h_over_R * R - scene.eps
    want = (h / R) ** 2
    for est in (NOREUSE, BIASED, UNBIASED):
        m, s = _image_mean_over_samples(orc, sc, AO, pos, nrm, pattern, est, 48, seed=21,
                                        radius=R)
        assert abs(m - want) < 4 * s + 1e-12, (est, m, want, s)
    # every reused occluder lies on the one plane, so Occ = 1 and biased == unbiased
    rec, _ = orc.trace(sc, AO, pos, nrm, radius=R, seed=21, sample=0)
    ob, mb = orc.reuse(sc, AO, pos, nrm, rec, pattern, BIASED, radius=R)
    ou, mu = orc.reuse(sc, AO, pos, nrm, rec, pattern, UNBIASED, radius=R)
    assert np.allclose(ob, ou, rtol=0, atol=1e-12)


@pytest.mark.parametrize("pattern", PATTERNS)
def test_shadow_fully_lit_is_one(orc, pattern):
    scene = synth.scene_plane_only()
    sc = orc.OracleScene(scene.tris)
    pos, nrm = _grid_case(scene)
    light = synth.light_c3().as_array()
    rec, _ = orc.trace(sc, SH, pos, nrm, light=light, seed=8, sample=0)
    assert np.all(rec[..., 7] < 0)
    for est in (NOREUSE, BIASED, UNBIASED, BOXMEAN):
        out, _ = orc.reuse(sc, SH, pos, nrm, rec, pattern, est, light=light)
        assert np.all(out == 1.0)
    out, _ = orc.reuse_light(sc, pos, pattern, light, seed=8, sample=0)
    assert np.all(out == 1.0)


@pytest.mark.parametrize("pattern", PATTERNS)
def test_shadow_fully_blocked(orc, pattern):
    scene = synth.scene_fully_blocked(2.0)
    sc = orc.OracleScene(scene.tris)
    pos, nrm = _grid_case(scene)
    light = synth.light_c3().as_array()
    for s in range(2):
        rec, _ = orc.trace(sc, SH, pos, nrm, light=light, seed=8, sample=s)
        assert np.all(rec[..., 7] >= 0)
        for est in (NOREUSE, BIASED, BOXMEAN):
            out, _ = orc.reuse(sc, SH, pos, nrm, rec, pattern, est, light=light)
            assert np.all(out == 0.0), est   # the guard makes the biased estimate exactly 0
        out, _ = orc.reuse_light(sc, pos, pattern, light, seed=8, sample=s)
        assert np.all(out == 0.0)
    m, s = _image_mean_over_samples(orc, sc, SH, pos, nrm, pattern, UNBIASED, 48, seed=8,
                                    light=light)
    assert abs(m) < 4 * s + 1e-12


def _half_plane_case():
    hb = 2.0
    scene = synth.scene_half_plane(hb)
    light = np.array([0.5, 0.0, 4.0, 1.0, 0, 0, 0, -0.5, 0], dtype=np.float32)
    W, H = 32, 2
    pos, nrm = synth.receiver_grid(W, H, 0.045, z=scene.eps, origin=(-0.5, 0.0))
    x = pos[..., 0].astype(np.float64)
    zr = float(pos[0, 0, 2])
    lam = (hb - zr) / (4.0 - zr)
    xstar = -x * (1 - lam) / lam
    want = np.clip((xstar - 0.0) / 1.0, 0.0, 1.0)
    return scene, light, pos, nrm, want


@pytest.mark.parametrize("est", [NOREUSE, UNBIASED, 4])
def test_shadow_half_plane_closed_form(orc, est):
    """Half-plane blocker: Shadow(x) = clamp((X* - a) / w, 0, 1), per pixel, in expectation."""
    scene, light, pos, nrm, want = _half_plane_case()
    sc = orc.OracleScene(scene.tris)
    M = 1024
    mean, var = orc.accumulate(sc, SH, pos, nrm, (BOX, 3, 1, None), est, light=light, seed=13,
                               sample0=0, M=M)
    sig = np.sqrt(var / M) + 1e-9
    z = (mean - want) / sig
    assert np.all(np.abs(z) < 5.0), np.abs(z).max()
    assert abs((mean - want).mean()) < 3 * math.sqrt((var / M).mean() / want.size) * 3
    assert want.min() == 0.0 and want.max() == 1.0 and ((want > 0) & (want < 1)).sum() > 20


@pytest.mark.parametrize("effect", [AO, SH])
def test_k1_equals_noreuse(orc, effect):
    scene = synth.scene_c1()
    sc = orc.OracleScene(scene.tris)
    pos, nrm, _ = orc.gbuffer(sc, synth.camera_c1().as_array(), 64, 64, scene.eps)
    light = synth.light_c3().as_array()
    R = 1.0
    for s in range(4):
        rec, _ = orc.trace(sc, effect, pos, nrm, radius=R, light=light, seed=31, sample=s)
        ref, _ = orc.reuse(sc, effect, pos, nrm, rec, (OFFS, 0, 0, None), NOREUSE, radius=R,
                           light=light)
        assert set(np.unique(ref).tolist()) <= {0.0, 1.0}
        for pat in [(OFFS, 0, 0, None), (BOX, 1, 1, None), (GROUP, 1, 1, None), (RAND, 6, 0, 5)]:
            for est in (BIASED, UNBIASED, BOXMEAN):
                out, _ = orc.reuse(sc, effect, pos, nrm, rec, pat, est, radius=R, light=light,
                                   sample=s)
                diff = np.argwhere(out != ref)
                for py, px in diff:
                    # only a hit whose own density vanishes exactly may differ
                    r = rec[py, px]
                    p = orc.density(effect, r[:3], r[3:6], pos[py, px, :3].astype(float),
                                    nrm[py, px, :3].astype(float), radius=R, light=light)
                    assert p == 0.0 and ref[py, px] == 0.0 and out[py, px] == 1.0
                assert len(diff) <= 2


def test_light_reuse_k1_equals_noreuse(orc):
    """Unbiased light-sample reuse with N_i = {i}: the receiver's own light sample, i.e. the
    step-1 shadow ray, bit for bit."""
    scene = synth.scene_c1()
    sc = orc.OracleScene(scene.tris)
    pos, nrm, _ = orc.gbuffer(sc, synth.camera_c1().as_array(), 64, 64, scene.eps)
    light = synth.light_c3().as_array()
    for s in range(3):
        rec, _ = orc.trace(sc, SH, pos, nrm, light=light, seed=31, sample=s)
        ref, _ = orc.reuse(sc, SH, pos, nrm, rec, (GROUP, 1, 1, None), NOREUSE, light=light)
        assert 0.0 < ref[pos[..., 3] > 0].mean() < 1.0
        for pat in [(OFFS, 0, 0, None), (BOX, 1, 1, None), (GROUP, 1, 1, None)]:
            out, _ = orc.reuse_light(sc, pos, pat, light, seed=31, sample=s)
            assert np.array_equal(out, ref)


def test_light_reuse_decomposes_into_member_segments(orc):
    """Light(2U) on a 2x1 group is, per receiver, the mean of the visibility of its own light
    sample and of its partner's: the partner's sample point is rebuilt from the partner's
    step-1 ray (orc.ray) and the segment tested with the brute-force closest hit."""
    scene = synth.scene_half_plane(2.0)
    sc = orc.OracleScene(scene.tris)
    light = np.array([0.5, 0.0, 4.0, 1.0, 0, 0, 0, -0.5, 0], dtype=np.float32)
    pos, nrm = synth.receiver_grid(8, 1, 0.11, z=scene.eps, origin=(-0.4, 0.0))
    mixed = 0
    for s in range(48):
        out, _ = orc.reuse_light(sc, pos, (GROUP, 2, 1, None), light, seed=5, sample=s)
        for i in range(8):
            j = i ^ 1
            vis = []
            for k in (i, j):
                dv, tm = orc.ray(SH, pos[0, k], nrm[0, k], k, 0.0, light, 5, s)
                y = pos[0, k, :3].astype(np.float64) + dv * tm
                seg = y - pos[0, i, :3].astype(np.float64)
                L = np.linalg.norm(seg)
                tri, _, _ = sc.closest_hit(pos[0, i, :3].astype(np.float64)[None], (seg / L)[None],
                                           np.array([L]), brute=True)
                vis.append(1.0 if tri[0] < 0 else 0.0)
            assert out[0, i] == 0.5 * (vis[0] + vis[1]), (s, i, out[0, i], vis)
            mixed += vis[0] != vis[1]
    assert mixed > 10          # the penumbra makes the two segments disagree often


@pytest.mark.parametrize("effect", [AO, SH])
@pytest.mark.parametrize("est", [BIASED, UNBIASED])
def test_mis_weights_sum_to_one(orc, effect, est):
    """Balance heuristic (Eq. 11): sum_k w_k(z_j) = 1 for every candidate with P_j > 0."""
    scene = synth.scene_c1()
    sc = orc.OracleScene(scene.tris)
    pos, nrm, _ = orc.gbuffer(sc, synth.camera_c1().as_array(), 64, 64, scene.eps)
    light = np.array([0.0, 0.0, 3.0, 4.0, 0, 0, 0, -4.0, 0], dtype=np.float32)
    rec, _ = orc.trace(sc, effect, pos, nrm, radius=1.0, light=light, seed=3, sample=0)
    rows = 0
    for pat in PATTERNS:
        for py in range(4, 60, 5):
            for px in range(4, 60, 5):
                if pos[py, px, 3] == 0:
                    continue
                mem, w = orc.mis_weights(sc, effect, pos, nrm, rec, pat, est, px, py, radius=1.0,
                                         light=light)
                s = w.sum(axis=1)
                nz = s > 0
                assert np.allclose(s[nz], 1.0, atol=1e-12)
                assert np.all(w >= 0)
                rows += nz.sum()
    assert rows > 200


# --------------------------------------------------------------------------------------
# Convergence of the unbiased estimators to a high-spp no-reuse reference
# --------------------------------------------------------------------------------------

def _convergence(orc, effect, pattern, M, region, light=None, R=1.0):
    scene = synth.scene_c1()
    sc = orc.OracleScene(scene.tris)
    pos, nrm, _ = orc.gbuffer(sc, synth.camera_c1().as_array(), 64, 64, scene.eps)
    mu, vu = orc.accumulate(sc, effect, pos, nrm, pattern, UNBIASED, radius=R, light=light,
                            seed=77, sample0=0, M=M, region=region)
    mr, vr = orc.accumulate(sc, effect, pos, nrm, (OFFS, 0, 0, None), NOREUSE, radius=R,
                            light=light, seed=77, sample0=1_000_000, M=M, region=region)
    sig = np.sqrt(vu / M + vr / M) + 1e-12
    z = (mu - mr) / sig
    assert np.all(np.abs(z) < 5.0), np.abs(z).max()
    bias = (mu - mr).mean()
    assert abs(bias) < 3 * math.sqrt((sig ** 2).mean() / z.size)
    assert ((mr > 0.05) & (mr < 0.95)).mean() > 0.5
    return mu, vu, mr, vr


@pytest.mark.slow
@pytest.mark.parametrize("pattern", [(GROUP, 2, 2, None), (BOX, 3, 3, None),
                                     (OFFS, 0, 0, synth.disk_offsets(8, 4.0, seed=9)),
                                     (RAND, 4, 7, 99)])
def test_unbiased_ao_converges_to_reference(orc, pattern):
    _convergence(orc, AO, pattern, 4096, (2, 44, 8, 8))


@pytest.mark.slow
@pytest.mark.parametrize("pattern", [(GROUP, 4, 2, None), (BOX, 3, 3, None)])
def test_unbiased_shadow_converges_to_reference(orc, pattern):
    light = np.array([0.0, 0.5, 3.0, 3.0, 0, 0, 0, -3.0, 0], dtype=np.float32)
    _convergence(orc, SH, pattern, 4096, (28, 20, 8, 8), light=light)
