"""Seeded synthetic scenes, G-buffers and initial parameters.

Stand-ins for the paper's scenes (Kitchen, Sponza, ...), which are not
available: the shapes follow the paper's workloads (1920x1080 frames, 32
point lights, a few dozen occluders, 8192 training positions), the
geometry is analytic.  All generators use numpy's PCG64 seeded explicitly,
compute in float64 and hand out float32 arrays; nothing here evaluates the
method (no encoding, MLP, visibility, sampling or shading).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

from .configs import NVCConfig, param_layout


@dataclass
class Scene:
    lights: np.ndarray      # float32 [L, 4]  x, y, z, intensity
    spheres: np.ndarray     # float32 [S, 4]  cx, cy, cz, r
    boxes: np.ndarray       # float32 [Bx, 6] lo xyz, hi xyz
    world_min: np.ndarray   # float32 [3] bounds of world-space training samples
    world_max: np.ndarray   # float32 [3]

    @property
    def n_lights(self) -> int:
        return int(self.lights.shape[0])


@dataclass
class GBuffer:
    pos: np.ndarray         # float32 [P, 3]
    nrm: np.ndarray         # float32 [P, 3] unit length
    width: int
    height: int

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def _unit_vectors(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def scene_unit_cube(seed: int = 0, n_lights: int = 4, n_spheres: int = 4,
                    intensity=(0.5, 2.0), radius=(0.05, 0.15)) -> Scene:
    """Point lights and sphere occluders uniform in the unit cube."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lp = rng.uniform(0.0, 1.0, (n_lights, 3))
    li = rng.uniform(intensity[0], intensity[1], (n_lights, 1))
    sc = rng.uniform(0.0, 1.0, (n_spheres, 3))
    sr = rng.uniform(radius[0], radius[1], (n_spheres, 1))
    return Scene(lights=_f32(np.hstack([lp, li])),
                 spheres=_f32(np.hstack([sc, sr])),
                 boxes=np.zeros((0, 6), np.float32),
                 world_min=_f32([0, 0, 0]), world_max=_f32([1, 1, 1]))


def gbuffer_points(seed: int, width: int, height: int,
                   lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> GBuffer:
    """Shading points uniform in a box with normals uniform on the sphere.

    Random normals make some lights face away (zero contribution), so the
    zero-weight paths of the sampler are exercised.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = width * height
    pos = rng.uniform(np.asarray(lo), np.asarray(hi), (n, 3))
    nrm = _unit_vectors(rng, n)
    return GBuffer(_f32(pos), _f32(nrm), width, height)


def gbuffer_camera_path(seed: int, frame: int, n_frames: int = 1000,
                        width: int = 64, height: int = 64) -> GBuffer:
    """The view at ``frame`` of a camera path through the unit-cube scene.

    The view is width*height points uniform in a cube of side 0.5 whose
    centre moves on a circle of radius 0.2 around (0.5, 0.5, 0.5) with a
    period of ``n_frames`` frames.
    """
    ang = 2.0 * np.pi * (frame % n_frames) / n_frames
    c = np.array([0.5 + 0.2 * np.cos(ang), 0.5 + 0.2 * np.sin(ang), 0.5])
    return gbuffer_points(seed * 1_000_003 + frame, width, height,
                          lo=tuple(c - 0.25), hi=tuple(c + 0.25))


class _Heightfield:
    """h(x, y) = 2 + sum_k a_k sin(f_k x + phi_k) sin(g_k y + psi_k), plus
    axis-aligned boxes standing on it (visible height = max of both)."""

    def __init__(self, rng: np.random.Generator, n_terms: int = 8,
                 n_boxes: int = 16, extent: float = 10.0):
        self.a = rng.uniform(0.1, 0.5, n_terms)
        self.f = rng.uniform(0.3, 2.0, n_terms)
        self.g = rng.uniform(0.3, 2.0, n_terms)
        self.phi = rng.uniform(0.0, 2 * np.pi, n_terms)
        self.psi = rng.uniform(0.0, 2 * np.pi, n_terms)
        self.extent = extent
        cx = rng.uniform(0.5, extent - 0.5, n_boxes)
        cy = rng.uniform(0.5, extent - 0.5, n_boxes)
        hx = rng.uniform(0.2, 0.8, n_boxes)
        hy = rng.uniform(0.2, 0.8, n_boxes)
        top = self.height(cx, cy) + rng.uniform(0.5, 2.0, n_boxes)
        self.boxes = np.stack([cx - hx, cy - hy, cx + hx, cy + hy, top], 1)

    def height(self, x, y):
        x = np.asarray(x, np.float64)[..., None]
        y = np.asarray(y, np.float64)[..., None]
        return 2.0 + np.sum(self.a * np.sin(self.f * x + self.phi)
                            * np.sin(self.g * y + self.psi), axis=-1)

    def gradient(self, x, y):
        x = np.asarray(x, np.float64)[..., None]
        y = np.asarray(y, np.float64)[..., None]
        hx = np.sum(self.a * self.f * np.cos(self.f * x + self.phi)
                    * np.sin(self.g * y + self.psi), axis=-1)
        hy = np.sum(self.a * self.g * np.sin(self.f * x + self.phi)
                    * np.cos(self.g * y + self.psi), axis=-1)
        return hx, hy


def scene_heightfield(seed: int = 1, n_lights: int = 32, n_spheres: int = 32,
                      n_boxes: int = 32, extent: float = 10.0) -> Scene:
    """Lights and occluders of the heightfield scene in [0, extent]^3.

    Lights U([0,10]^2 x [4,10]) with intensity U(20, 100); sphere occluders
    with radius U(0.2, 0.8) and boxes with half-extent U(0.2, 1), centres in
    [0,10] x [0,10] x [3,9].  The heightfield itself (see
    ``gbuffer_heightfield``) only makes shading positions and normals.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    _Heightfield(rng, extent=extent)  # consume the same stream as the G-buffer
    lp = np.stack([rng.uniform(0, extent, n_lights),
                   rng.uniform(0, extent, n_lights),
                   rng.uniform(0.4 * extent, extent, n_lights)], 1)
    li = rng.uniform(20.0, 100.0, (n_lights, 1))
    sc = np.stack([rng.uniform(0, extent, n_spheres),
                   rng.uniform(0, extent, n_spheres),
                   rng.uniform(0.3 * extent, 0.9 * extent, n_spheres)], 1)
    sr = rng.uniform(0.2, 0.8, (n_spheres, 1))
    bc = np.stack([rng.uniform(0, extent, n_boxes),
                   rng.uniform(0, extent, n_boxes),
                   rng.uniform(0.3 * extent, 0.9 * extent, n_boxes)], 1)
    bh = rng.uniform(0.2, 1.0, (n_boxes, 3))
    return Scene(lights=_f32(np.hstack([lp, li])),
                 spheres=_f32(np.hstack([sc, sr])),
                 boxes=_f32(np.hstack([bc - bh, bc + bh])),
                 world_min=_f32([0, 0, 0]),
                 world_max=_f32([extent, extent, extent]))


def scene_many_lights(seed: int = 1, n_lights: int = 1024, n_groups: int = 64,
                      n_spheres: int = 32, n_boxes: int = 32,
                      extent: float = 10.0) -> Scene:
    """Many-lights variant of the heightfield scene: the occluders of
    ``scene_heightfield(seed, n_lights=n_groups, ...)`` and ``n_lights``
    point lights in ``n_groups`` fixtures, each fixture's lights spread
    N(0, 0.25^2) per axis around the heightfield scene's light position
    (clipped to x, y in [0, extent], z in [0.4 extent, extent]).  Intensities
    U(20, 100) * 32 / n_lights keep the total power of 32 lights.  The
    fixtures give the lights the grouped structure (lamps, strips) that
    clustering exploits; the G-buffer is ``gbuffer_heightfield(seed)``."""
    base = scene_heightfield(seed, n_lights=n_groups, n_spheres=n_spheres,
                             n_boxes=n_boxes, extent=extent)
    rng = np.random.Generator(np.random.PCG64([seed, 7]))
    g = rng.integers(0, n_groups, n_lights)
    p = base.lights[g, :3].astype(np.float64) + rng.normal(0.0, 0.25, (n_lights, 3))
    p[:, :2] = np.clip(p[:, :2], 0.0, extent)
    p[:, 2] = np.clip(p[:, 2], 0.4 * extent, extent)
    li = rng.uniform(20.0, 100.0, (n_lights, 1)) * (32.0 / n_lights)
    return Scene(lights=_f32(np.hstack([p, li])), spheres=base.spheres,
                 boxes=base.boxes, world_min=base.world_min,
                 world_max=base.world_max)


def scene_rooms(seed: int = 1, n_lights: int = 1024, rooms: int = 4,
                fixtures_per_room: int = 2, n_spheres: int = 32, n_boxes: int = 32,
                extent: float = 10.0, wall: float = 0.08, door_width: float = 0.8,
                door_height: float = 5.0) -> Scene:
    """Interior of ``rooms`` x ``rooms`` rooms over the heightfield: the
    occluders of ``scene_heightfield(seed, ...)`` plus full-height walls
    (boxes ``wall`` thick on the lines x, y = i * extent / rooms) with a
    doorway ``door_width`` wide and ``door_height`` high in the middle of
    every room edge.  Each room has ``fixtures_per_room`` ceiling fixtures
    (x, y uniform 0.3 inside the room, z U(7, 9.5)); every light joins a
    uniformly drawn fixture with an N(0, 0.15^2) offset per axis (clipped
    0.1 inside its room, z in [4, 9.9]), intensity U(20, 100) * 32 / n_lights.
    Lights of other rooms are seen only through doorways: the many-rooms
    structure clustering exploits.  G-buffer: ``gbuffer_heightfield(seed)``."""
    base = scene_heightfield(seed, n_lights=1, n_spheres=n_spheres,
                             n_boxes=n_boxes, extent=extent)
    rng = np.random.Generator(np.random.PCG64([seed, 13]))
    s = extent / rooms
    n_fix = rooms * rooms * fixtures_per_room
    room = np.repeat(np.arange(rooms * rooms), fixtures_per_room)
    rx, ry = (room % rooms) * s, (room // rooms) * s
    fx = rx + rng.uniform(0.3, s - 0.3, n_fix)
    fy = ry + rng.uniform(0.3, s - 0.3, n_fix)
    fz = rng.uniform(7.0, 9.5, n_fix)
    g = rng.integers(0, n_fix, n_lights)
    p = np.stack([fx[g], fy[g], fz[g]], 1) + rng.normal(0.0, 0.15, (n_lights, 3))
    p[:, 0] = np.clip(p[:, 0], rx[g] + 0.1, rx[g] + s - 0.1)
    p[:, 1] = np.clip(p[:, 1], ry[g] + 0.1, ry[g] + s - 0.1)
    p[:, 2] = np.clip(p[:, 2], 4.0, 9.9)
    li = rng.uniform(20.0, 100.0, (n_lights, 1)) * (32.0 / n_lights)
    t, hw = 0.5 * wall, 0.5 * door_width
    walls = []
    for i in range(1, rooms):
        c = i * s
        for b in range(rooms):
            a0, a1, m = b * s, (b + 1) * s, (b + 0.5) * s
            for lo, hi in ((a0, m - hw), (m + hw, a1)):
                walls.append([c - t, lo, 0.0, c + t, hi, extent])     # wall along y
                walls.append([lo, c - t, 0.0, hi, c + t, extent])     # wall along x
            walls.append([c - t, m - hw, door_height, c + t, m + hw, extent])
            walls.append([m - hw, c - t, door_height, m + hw, c + t, extent])
    return Scene(lights=_f32(np.hstack([p, li])), spheres=base.spheres,
                 boxes=_f32(np.vstack([base.boxes, np.asarray(walls)])),
                 world_min=base.world_min, world_max=base.world_max)


def kmeans_init(n_lights: int, k: int, seed: int = 0) -> np.ndarray:
    """k distinct light indices drawn uniformly: the seeds of k-means."""
    rng = np.random.Generator(np.random.PCG64([seed, 11]))
    return rng.choice(n_lights, k, replace=False).astype(np.int32)


def gbuffer_heightfield(seed: int = 1, width: int = 1920, height: int = 1080,
                        extent: float = 10.0, window=None) -> GBuffer:
    """Orthographic top-down view of the heightfield + boxes.

    Pixel (i, j) looks straight down at (x, y) = window origin + ((j+0.5)/W,
    (i+0.5)/H) * window size; the visible point is the heightfield or, where
    a box covers (x, y) and its top is higher, the box top (normal +z).
    ``window`` = (x0, y0, size_x, size_y), default the whole [0, extent]^2.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    hf = _Heightfield(rng, extent=extent)
    x0, y0, sx, sy = window if window is not None else (0.0, 0.0, extent, extent)
    xs = x0 + (np.arange(width) + 0.5) / width * sx
    ys = y0 + (np.arange(height) + 0.5) / height * sy
    X, Y = np.meshgrid(xs, ys)           # [H, W], row i = y
    Z = hf.height(X, Y)
    gx, gy = hf.gradient(X, Y)
    N = np.stack([-gx, -gy, np.ones_like(gx)], -1)
    N /= np.linalg.norm(N, axis=-1, keepdims=True)
    for (bx0, by0, bx1, by1, top) in hf.boxes:
        m = (X >= bx0) & (X <= bx1) & (Y >= by0) & (Y <= by1) & (top > Z)
        Z = np.where(m, top, Z)
        N[m] = (0.0, 0.0, 1.0)
    pos = np.stack([X, Y, Z], -1).reshape(-1, 3)
    return GBuffer(_f32(pos), _f32(N.reshape(-1, 3)), width, height)


def multiview_gbuffers(seed: int = 0, sizes=((1280, 720), (1920, 1080),
                                             (2560, 1440), (3840, 2160))
                       ) -> List[GBuffer]:
    """Several views of the unit-cube scene at uneven resolutions."""
    return [gbuffer_points(seed * 7919 + 17 * v + 1, w, h)
            for v, (w, h) in enumerate(sizes)]


def init_params(cfg: NVCConfig, seed: int = 0) -> np.ndarray:
    """Initial parameter vector (float32), laid out as ``param_layout``.

    Table entries ~ U(-a, a) with a = cfg.table_init.  Weights: Xavier
    uniform, U(+-sqrt(6 / (n_in + n_out))), or He normal, N(0, 2 / n_in)
    (Section 3.4 uses He).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t_off, t_n, layers = param_layout(cfg)
    total = t_n + sum(o * i for _, o, i in layers)
    p = np.empty(total, np.float64)
    p[t_off:t_off + t_n] = rng.uniform(-cfg.table_init, cfg.table_init, t_n)
    for off, n_out, n_in in layers:
        if cfg.init == "xavier_uniform":
            a = np.sqrt(6.0 / (n_in + n_out))
            w = rng.uniform(-a, a, n_out * n_in)
        elif cfg.init == "he_normal":
            w = rng.standard_normal(n_out * n_in) * np.sqrt(2.0 / n_in)
        else:
            raise ValueError(cfg.init)
        p[off:off + n_out * n_in] = w
    return p.astype(np.float32)
