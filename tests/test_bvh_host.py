"""The BVH builder on the CPU (occ_debug_bvh_host: the same build as occ_bvh_build, without a
device): every triangle sits in exactly one leaf with its input id, every child box holds
all triangles below it, the tree fits the traversal stack, and a stack traversal of the tree
in FP64 finds the same closest hit as brute force over all triangles for short and long rays.
The scenes are the small box scene and a reduced terrain with boxes and spheres, whose
binary tree is collapsed into 4-wide nodes by the surface-area dynamic program."""
import numpy as np
import pytest

import synth

EMPTY = 0x7FFFFFFF
LEAF = 0x80000000


def _decode(nodes):
    planes = nodes[:, :24].reshape(-1, 6, 4).astype(np.float64)   # [N, plane, child]
    refs = nodes[:, 24:28].copy().view(np.uint32)
    return planes, refs


def _leaf(ref):
    return int(ref) & 0x3FFFFFF, ((int(ref) & 0x7FFFFFFF) >> 26) + 1


def _hit_t(v, o, d, tmax):
    """Moller-Trumbore in FP64 for every triangle of v [T, 3, 3]: t on (0, tmax] or inf."""
    e1, e2 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]
    p = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, p)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / det
        s = o - v[:, 0]
        u = np.einsum("ij,ij->i", s, p) * inv
        q = np.cross(s, e1)
        w = (q @ d) * inv
        t = np.einsum("ij,ij->i", e2, q) * inv
    ok = (np.abs(det) > 1e-300) & (u >= 0) & (u <= 1) & (w >= 0) & (u + w <= 1) & (t > 0) & (t <= tmax)
    return np.where(ok, t, np.inf)


@pytest.mark.parametrize("which", ["c1", "terrain"])
def test_host_bvh_is_complete_and_finds_the_closest_hits(which):
    from paper_2607_23122_gb300 import occ
    if which == "c1":
        tris = synth.scene_c1().tris
    else:
        tris = synth.scene_terrain(grid=96, n_spheres=30, n_boxes=400, seed=5).tris
    tris = np.asarray(tris, dtype=np.float32)
    T = tris.shape[0]
    nodes, tout, depth = occ.occ_debug_bvh_host(tris)
    planes, refs = _decode(nodes)
    assert 3 * (depth) <= 64                            # three pushes per level fit the stack
    ids = tout[:, 3].copy().view(np.uint32)
    assert np.array_equal(np.sort(ids), np.arange(T, dtype=np.uint32))
    verts = tout[:, [0, 1, 2, 4, 5, 6, 8, 9, 10]].reshape(-1, 3, 3)
    assert np.array_equal(verts, tris[ids])             # leaf-order copy of the input
    # every triangle in exactly one leaf; child boxes hold their subtrees
    seen = np.zeros(T, dtype=np.int64)

    def subtree(ref):
        """(lo, hi) of everything below ref; asserts containment on the way."""
        if ref & LEAF:
            first, cnt = _leaf(ref)
            seen[first:first + cnt] += 1
            v = verts[first:first + cnt].reshape(-1, 3)
            return v.min(0), v.max(0)
        lo, hi = np.full(3, np.inf), np.full(3, -np.inf)
        for c in range(4):
            r = int(refs[ref, c])
            if r == EMPTY:
                assert np.all(planes[ref, 0::2, c] == np.inf) and np.all(planes[ref, 1::2, c] == -np.inf)
                continue
            clo, chi = subtree(r)
            assert np.all(planes[ref, 0::2, c] <= clo) and np.all(planes[ref, 1::2, c] >= chi)
            lo, hi = np.minimum(lo, clo), np.maximum(hi, chi)
        return lo, hi

    import sys
    old = sys.getrecursionlimit()
    sys.setrecursionlimit(max(old, 10000))
    try:
        subtree(0)
    finally:
        sys.setrecursionlimit(old)
    assert np.all(seen == 1)
    # closest hits: FP64 stack traversal of the tree against brute force
    rng = np.random.default_rng(17)
    v64 = verts.astype(np.float64)
    mism = 0
    for k in range(150):
        i = rng.integers(T)
        o = v64[i].mean(0) + 0.01 * (rng.random(3) - 0.5)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        tmax = 0.5 if k % 2 == 0 else 50.0
        want = _hit_t(v64, o, d, tmax).min()
        got, stack = np.inf, [0]
        while stack:
            ref = stack.pop()
            if ref & LEAF:
                first, cnt = _leaf(ref)
                got = min(got, _hit_t(v64[first:first + cnt], o, d, tmax).min())
                continue
            for c in range(4):
                r = int(refs[ref, c])
                if r == EMPTY:
                    continue
                t0, t1 = 0.0, tmax
                for a in range(3):
                    lo, hi = planes[ref, 2 * a, c], planes[ref, 2 * a + 1, c]
                    if d[a] == 0.0:
                        if o[a] < lo or o[a] > hi:
                            t0 = np.inf
                        continue
                    ta, tb = (lo - o[a]) / d[a], (hi - o[a]) / d[a]
                    t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
                if t0 <= t1:
                    stack.append(r)
        # the same FP64 test on a subset can round its last bit differently (vectorised sums)
        mism += not (got == want or abs(got - want) <= 1e-12 * max(1.0, want))
    assert mism == 0
