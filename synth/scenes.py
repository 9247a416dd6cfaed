"""Procedural scenes, cameras, lights and neighbour patterns (input data only).

The paper evaluates on Falcor assets that are not available here, so these
seeded generators stand in for them with the same structure: a ground surface
with many small closed objects resting on it, seen by a pinhole camera, lit by
one rectangular area light (Sec. 5, Sec. 6).  Every random choice comes from
NumPy's Philox bit generator seeded with the scene seed, so a seed fixes the
scene bit for bit on any machine.

Conventions: +z is up, triangles are float32 arrays of shape [T, 3, 3]
(triangle, vertex, xyz).  ``eps`` is the receiver offset along the surface
normal, 1e-4 of the scene bounding-box diagonal.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Camera:
    eye: tuple
    target: tuple
    vfov_deg: float
    up: tuple = (0.0, 0.0, 1.0)

    def as_array(self) -> np.ndarray:
        """[eye(3), target(3), up(3), vfov_deg] as float32."""
        return np.array(list(self.eye) + list(self.target) + list(self.up) + [self.vfov_deg],
                        dtype=np.float32)


@dataclasses.dataclass
class RectLight:
    """Rectangle c + a*eu + b*ev, a, b in [-1/2, 1/2]; emits along normalize(eu x ev)."""
    c: tuple
    eu: tuple
    ev: tuple

    def as_array(self) -> np.ndarray:
        return np.array(list(self.c) + list(self.eu) + list(self.ev), dtype=np.float32)


@dataclasses.dataclass
class Scene:
    name: str
    tris: np.ndarray          # float32 [T, 3, 3]
    eps: float                # receiver offset along the normal

    @property
    def num_tris(self) -> int:
        return int(self.tris.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def _finish(name: str, tris: np.ndarray) -> Scene:
    tris = np.ascontiguousarray(tris, dtype=np.float32)
    lo = tris.reshape(-1, 3).min(axis=0).astype(np.float64)
    hi = tris.reshape(-1, 3).max(axis=0).astype(np.float64)
    eps = float(np.float32(1e-4 * np.linalg.norm(hi - lo)))
    return Scene(name=name, tris=tris, eps=eps)


def _quad(p0, p1, p2, p3) -> np.ndarray:
    """Two triangles for the quad p0 p1 p2 p3 (counter-clockwise)."""
    return np.array([[p0, p1, p2], [p0, p2, p3]], dtype=np.float64)


_BOX_FACES = np.array([
    [0, 2, 1], [0, 3, 2],      # bottom (z-)
    [4, 5, 6], [4, 6, 7],      # top (z+)
    [0, 1, 5], [0, 5, 4],      # y-
    [1, 2, 6], [1, 6, 5],      # x+
    [2, 3, 7], [2, 7, 6],      # y+
    [3, 0, 4], [3, 4, 7],      # x-
], dtype=np.int64)


def _boxes(centers_xy, half_xy, z0, z1, yaw) -> np.ndarray:
    """Oriented boxes: centre (x, y), half extents (hx, hy), z range, yaw -> [n*12, 3, 3]."""
    n = centers_xy.shape[0]
    sx = np.array([-1, 1, 1, -1], dtype=np.float64)
    sy = np.array([-1, -1, 1, 1], dtype=np.float64)
    lx = sx[None, :] * half_xy[:, 0:1]
    ly = sy[None, :] * half_xy[:, 1:2]
    c, s = np.cos(yaw)[:, None], np.sin(yaw)[:, None]
    wx = centers_xy[:, 0:1] + c * lx - s * ly
    wy = centers_xy[:, 1:2] + s * lx + c * ly
    corners = np.zeros((n, 8, 3))
    corners[:, :4, 0] = wx
    corners[:, :4, 1] = wy
    corners[:, :4, 2] = z0[:, None]
    corners[:, 4:, 0] = wx
    corners[:, 4:, 1] = wy
    corners[:, 4:, 2] = z1[:, None]
    return corners[:, _BOX_FACES, :].reshape(-1, 3, 3)


def _icosphere(subdiv: int) -> np.ndarray:
    """Unit icosphere as a triangle array [20 * 4**subdiv, 3, 3]."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    return V[np.array(faces)]


# --------------------------------------------------------------------------------------
# Small scene: ground quad + 16 boxes (about 200 triangles)
# --------------------------------------------------------------------------------------

def scene_c1(seed: int = 1, n_boxes: int = 16) -> Scene:
    """Ground quad [-4, 4]^2 at z = 0 plus ``n_boxes`` random boxes resting on it."""
    rng = _rng(seed)
    ground = _quad((-4, -4, 0), (4, -4, 0), (4, 4, 0), (-4, 4, 0))
    centers = rng.uniform(-2.5, 2.5, size=(n_boxes, 2))
    half = rng.uniform(0.15, 0.6, size=(n_boxes, 2))
    heights = rng.uniform(0.2, 1.5, size=n_boxes)
    yaw = rng.uniform(0.0, math.pi / 2, size=n_boxes)
    boxes = _boxes(centers, half, np.zeros(n_boxes), heights, yaw)
    return _finish(f"c1_seed{seed}", np.concatenate([ground, boxes]))


def camera_c1() -> Camera:
    return Camera(eye=(0.0, -6.0, 4.5), target=(0.0, 0.0, 0.3), vfov_deg=50.0)


# --------------------------------------------------------------------------------------
# Large scene: heightfield + icospheres + boxes (about 1M or 4M triangles)
# --------------------------------------------------------------------------------------

def _height_fn(rng: np.random.Generator, n_waves: int = 8, amplitude: float = 0.8):
    w = rng.uniform(0.3, 1.0, size=n_waves)
    amp = amplitude * w / w.sum()
    ang = rng.uniform(0.0, 2 * math.pi, size=n_waves)
    lam = rng.uniform(2.5, 12.0, size=n_waves)
    kx = 2 * math.pi / lam * np.cos(ang)
    ky = 2 * math.pi / lam * np.sin(ang)
    ph = rng.uniform(0.0, 2 * math.pi, size=n_waves)

    def h(x, y):
        x = np.asarray(x, dtype=np.float64)[..., None]
        y = np.asarray(y, dtype=np.float64)[..., None]
        return (amp * np.sin(kx * x + ky * y + ph)).sum(axis=-1)

    return h


def scene_terrain(grid: int = 512, extent: float = 16.0, n_spheres: int = 300,
                  n_boxes: int = 8000, seed: int = 2, sphere_subdiv: int = 3) -> Scene:
    """Heightfield over [-extent, extent]^2 with icospheres and boxes resting on it.

    grid=512, 300 spheres, 8000 boxes gives 522,242 + 384,000 + 96,000 = 1,002,242
    triangles; grid=1024, 1200 spheres, 30000 boxes gives about 3.99M.
    """
    rng = _rng(seed)
    h = _height_fn(rng)
    xs = np.linspace(-extent, extent, grid)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    Z = h(X, Y)
    P = np.stack([X, Y, Z], axis=-1)
    a = P[:-1, :-1].reshape(-1, 3)
    b = P[:-1, 1:].reshape(-1, 3)
    c = P[1:, 1:].reshape(-1, 3)
    d = P[1:, :-1].reshape(-1, 3)
    terrain = np.empty((2 * a.shape[0], 3, 3))
    terrain[0::2] = np.stack([a, b, c], axis=1)
    terrain[1::2] = np.stack([a, c, d], axis=1)

    margin = 1.0
    sc = rng.uniform(-extent + margin, extent - margin, size=(n_spheres, 2))
    sr = rng.uniform(0.15, 0.6, size=n_spheres)
    unit = _icosphere(sphere_subdiv)
    sz = h(sc[:, 0], sc[:, 1]) + sr * 0.9
    spheres = (unit[None] * sr[:, None, None, None]
               + np.stack([sc[:, 0], sc[:, 1], sz], axis=-1)[:, None, None, :]).reshape(-1, 3, 3)

    bc = rng.uniform(-extent + margin, extent - margin, size=(n_boxes, 2))
    bh = rng.uniform(0.05, 0.4, size=(n_boxes, 3))
    yaw = rng.uniform(0.0, math.pi / 2, size=n_boxes)
    z0 = h(bc[:, 0], bc[:, 1]) - 0.3 * bh[:, 2]
    boxes = _boxes(bc, bh[:, :2], z0, z0 + 2 * bh[:, 2], yaw)
    return _finish(f"terrain{grid}_seed{seed}", np.concatenate([terrain, spheres, boxes]))


def camera_c2() -> Camera:
    return Camera(eye=(0.0, -14.0, 6.0), target=(0.0, 0.0, 0.0), vfov_deg=55.0)


def light_c3() -> RectLight:
    """1 x 0.5 rectangle at height 4 facing down (eu x ev points to -z)."""
    return RectLight(c=(0.0, 0.0, 4.0), eu=(1.0, 0.0, 0.0), ev=(0.0, -0.5, 0.0))


def serving_views(n: int = 8) -> list:
    """Preset cameras around the terrain scene (request mix of the serving loop)."""
    views = []
    for i in range(n):
        ang = 2 * math.pi * i / n - math.pi / 2
        r = 14.0 - 2.0 * (i % 2)
        views.append(Camera(eye=(r * math.cos(ang), r * math.sin(ang), 5.0 + (i % 3)),
                            target=(0.0, 0.0, 0.0), vfov_deg=55.0))
    return views


# --------------------------------------------------------------------------------------
# Closed-form scenes with directly synthesized receivers
# --------------------------------------------------------------------------------------

def receiver_grid(W: int, H: int, spacing: float, z: float = 0.0,
                  origin=(0.0, 0.0)) -> tuple:
    """G-buffer of a W x H grid of receivers on the plane at height ``z``, normal +z.

    Pixel (px, py) sits at origin + ((px - (W-1)/2) * spacing, (py - (H-1)/2) * spacing).
    Returns float32 arrays pos4 [H, W, 4] (w = 1 marks a valid receiver) and nrm4.
    """
    px = (np.arange(W) - (W - 1) / 2.0) * spacing + origin[0]
    py = (np.arange(H) - (H - 1) / 2.0) * spacing + origin[1]
    X, Y = np.meshgrid(px, py, indexing="xy")
    pos = np.zeros((H, W, 4), dtype=np.float32)
    pos[..., 0] = X
    pos[..., 1] = Y
    pos[..., 2] = z
    pos[..., 3] = 1.0
    nrm = np.zeros((H, W, 4), dtype=np.float32)
    nrm[..., 2] = 1.0
    return pos, nrm


def scene_plane_only(half: float = 50.0) -> Scene:
    """The receiving floor alone (z = 0): nothing can occlude a receiver above it."""
    return _finish("plane_only", _quad((-half, -half, 0), (half, -half, 0),
                                       (half, half, 0), (-half, half, 0)))


def scene_parallel_plane(height: float, half: float = 50.0) -> Scene:
    """An occluding plane at z = ``height`` above a receiving floor at z = 0."""
    floor = _quad((-half, -half, 0), (half, -half, 0), (half, half, 0), (-half, half, 0))
    top = _quad((-half, -half, height), (-half, half, height),
                (half, half, height), (half, -half, height))
    return _finish(f"parallel_plane_h{height}", np.concatenate([floor, top]))


def scene_half_plane(blocker_height: float, half: float = 50.0) -> Scene:
    """Floor at z = 0 and a blocker half-plane {X >= 0} at z = ``blocker_height``."""
    floor = _quad((-half, -half, 0), (half, -half, 0), (half, half, 0), (-half, half, 0))
    blk = _quad((0.0, -half, blocker_height), (half, -half, blocker_height),
                (half, half, blocker_height), (0.0, half, blocker_height))
    return _finish(f"half_plane_h{blocker_height}", np.concatenate([floor, blk]))


def scene_fully_blocked(blocker_height: float = 2.0, half: float = 50.0) -> Scene:
    """Floor plus a large plane between every receiver and the light."""
    return scene_parallel_plane(blocker_height, half)


# --------------------------------------------------------------------------------------
# Neighbour patterns
# --------------------------------------------------------------------------------------

def disk_offsets(K: int, radius: float = 15.0, seed: int = 3) -> np.ndarray:
    """K-1 distinct pixel offsets (dx, dy) != (0, 0) drawn uniformly from the disk.

    The receiver itself is the K-th member of its neighbour set; the offsets are
    shared by every pixel of a frame.  Returns int32 [K-1, 2].
    """
    r = int(math.floor(radius))
    cand = [(dx, dy) for dy in range(-r, r + 1) for dx in range(-r, r + 1)
            if (dx or dy) and dx * dx + dy * dy <= radius * radius]
    rng = _rng(seed)
    idx = rng.choice(len(cand), size=K - 1, replace=False)
    return np.array([cand[i] for i in sorted(idx)], dtype=np.int32).reshape(K - 1, 2)
