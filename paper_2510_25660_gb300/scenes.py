"""Seeded synthetic scene generators (inputs only).

These functions build triangle soups, per-triangle materials, emitters, cameras,
relay-wall scan grids and density grids with numpy's PCG64.  They hold none of
the rendering arithmetic: both the CUDA path and the CPU oracle consume the flat
arrays they return.  The paper's own scenes (Staircase, Bottle, Office, the
Cornell box of its usage listing in Sec. 2) are not available, so these are
stand-ins with the shapes of the paper's workloads: a Cornell box about 2 m wide
(Sec. 2 listing, Sec. 4.3 figure), a large procedural scene, a relay wall with a
hidden mesh (Sec. 4.5), and a box filled with a heterogeneous medium (Sec. 4.1).

Conventions shared by every consumer:
  * triangles: float32 [N, 3, 3] (vertex, xyz); the geometric normal of a
    triangle is (v1 - v0) x (v2 - v0); emitters emit from that side only.
  * materials: albedo float32 [N, 3], roughness float32 [N], mtype uint32 [N]
    (0 = Lambertian with albedo rho, 1 = GGX conductor with F0 = albedo).
  * emitters: list of dicts {type: 0 area | 1 point, first_tri, n_tris,
    radiance (RGB; intensity W/sr for points), position (points only)}.
  * camera: origin, target, up, fov_x_deg (horizontal field of view).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

LAMBERT = 0
GGX = 1
EMITTER_AREA = 0
EMITTER_POINT = 1

SCENE_SEED = 2510
RENDER_SEED = 25660
TARGET_SEED = 25661


@dataclasses.dataclass
class Scene:
    tris: np.ndarray                 # float32 [N,3,3]
    albedo: np.ndarray               # float32 [N,3]
    roughness: np.ndarray            # float32 [N]
    mtype: np.ndarray                # uint32 [N]
    emitters: list                   # list of dict
    camera: dict                     # origin/target/up/fov_x_deg
    medium: Optional[dict] = None    # lo, hi, density [R,R,R] float32, albedo, g
    hidden: Optional[tuple] = None   # (first_tri, n_tris) of the NLOS hidden mesh
    wall: Optional[dict] = None      # NLOS relay wall: center, size, normal, albedo

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


@dataclasses.dataclass
class FilmSpec:
    H: int
    W: int
    T: int
    C: int
    start_opl: float
    bin_width: float


# ----------------------------------------------------------------------------
# primitive meshes
# ----------------------------------------------------------------------------

def quad(p0, p1, p2, p3) -> np.ndarray:
    """Two triangles (p0,p1,p2), (p0,p2,p3); normal follows (p1-p0)x(p2-p0)."""
    p0, p1, p2, p3 = (np.asarray(p, np.float64) for p in (p0, p1, p2, p3))
    return np.stack([np.stack([p0, p1, p2]), np.stack([p0, p2, p3])])


def box_mesh(center, size, rot_y_deg: float, inward: bool = False) -> np.ndarray:
    """Axis box of the given size, rotated about +y, 12 triangles, normals out."""
    hx, hy, hz = (0.5 * s for s in size)
    c = np.array([[-hx, -hy, -hz], [hx, -hy, -hz], [hx, hy, -hz], [-hx, hy, -hz],
                  [-hx, -hy, hz], [hx, -hy, hz], [hx, hy, hz], [-hx, hy, hz]])
    faces = [(4, 5, 6, 7),   # +z
             (1, 0, 3, 2),   # -z
             (5, 1, 2, 6),   # +x
             (0, 4, 7, 3),   # -x
             (7, 6, 2, 3),   # +y
             (0, 1, 5, 4)]   # -y
    a = math.radians(rot_y_deg)
    R = np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])
    v = c @ R.T + np.asarray(center, np.float64)
    out = []
    for f in faces:
        q = quad(v[f[0]], v[f[1]], v[f[2]], v[f[3]])
        if inward:
            q = q[:, ::-1, :]
        out.append(q)
    return np.concatenate(out)


def icosphere(level: int) -> np.ndarray:
    """Unit icosphere as a triangle soup of 20*4^level outward-wound triangles."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]])
    tri = v[f]
    for _ in range(level):
        a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]
        ab = a + b
        bc = b + c
        ca = c + a
        ab /= np.linalg.norm(ab, axis=1, keepdims=True)
        bc /= np.linalg.norm(bc, axis=1, keepdims=True)
        ca /= np.linalg.norm(ca, axis=1, keepdims=True)
        tri = np.concatenate([np.stack([a, ab, ca], 1), np.stack([ab, b, bc], 1),
                              np.stack([ca, bc, c], 1), np.stack([ab, bc, ca], 1)])
    # make the winding outward: (v1-v0)x(v2-v0) . centroid > 0
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    flip = np.einsum("ij,ij->i", n, tri.mean(1)) < 0
    tri[flip] = tri[flip][:, ::-1]
    return tri


# ----------------------------------------------------------------------------
# seeded value noise (lattice values from PCG64, smoothstep interpolation)
# ----------------------------------------------------------------------------

class ValueNoise:
    def __init__(self, seed: int, dim: int, period: int = 64):
        self.P = period
        self.dim = dim
        self.table = np.random.default_rng(seed).random((period,) * dim)

    @staticmethod
    def _s(f):
        return f * f * (3.0 - 2.0 * f)

    def __call__(self, *coords):
        P = self.P
        i = [np.floor(c).astype(np.int64) for c in coords]
        f = [self._s(c - np.floor(c)) for c in coords]
        out = 0.0
        for corner in range(1 << self.dim):
            w = 1.0
            idx = []
            for d in range(self.dim):
                bit = (corner >> d) & 1
                w = w * (f[d] if bit else (1.0 - f[d]))
                idx.append((i[d] + bit) % P)
            out = out + w * self.table[tuple(idx)]
        return out

    def fbm(self, *coords, octaves=5, lacunarity=2.0, gain=0.5):
        amp, tot, norm = 1.0, 0.0, 0.0
        freq = 1.0
        for _ in range(octaves):
            tot = tot + amp * self(*[c * freq for c in coords])
            norm += amp
            amp *= gain
            freq *= lacunarity
        return tot / norm  # in [0, 1]


# ----------------------------------------------------------------------------
# scene builders
# ----------------------------------------------------------------------------

def _assemble(parts, rng=None):
    tris = np.concatenate([p[0] for p in parts]).astype(np.float32)
    albedo = np.concatenate([np.broadcast_to(np.asarray(p[1], np.float32), (len(p[0]), 3)) for p in parts])
    rough = np.concatenate([np.full(len(p[0]), p[2], np.float32) for p in parts])
    mtype = np.concatenate([np.full(len(p[0]), p[3], np.uint32) for p in parts])
    return tris, np.ascontiguousarray(albedo, np.float32), rough, mtype


def cornell_box(seed: int = SCENE_SEED) -> Scene:
    """36-triangle Cornell box: [-1,1]^3 with the +z face open, two blocks, one
    0.5 m ceiling quad light of radiance 10 facing down, camera 3.5 m away."""
    rng = np.random.default_rng(seed)
    L = -1.0
    H = 1.0
    walls = [
        quad((L, L, H), (H, L, H), (H, L, L), (L, L, L)),        # floor  (normal +y)
        quad((L, H, L), (H, H, L), (H, H, H), (L, H, H)),        # ceiling (normal -y)
        quad((L, L, L), (H, L, L), (H, H, L), (L, H, L)),        # back   (normal +z)
        quad((L, L, H), (L, L, L), (L, H, L), (L, H, H)),        # left   (normal +x)
        quad((H, L, L), (H, L, H), (H, H, H), (H, H, L)),        # right  (normal -x)
    ]
    parts = []
    for w in walls:
        parts.append((w, rng.uniform(0.2, 0.8, 3), 0.0, LAMBERT))
    short = box_mesh((0.35, -0.7, 0.3), (0.6, 0.6, 0.6), 15.0)
    tall = box_mesh((-0.35, -0.4, -0.3), (0.6, 1.2, 0.6), -15.0)
    for blk in (short, tall):
        for q in range(6):
            parts.append((blk[2 * q:2 * q + 2], rng.uniform(0.2, 0.8, 3), 0.0, LAMBERT))
    y = 0.999
    light = quad((-0.25, y, -0.25), (0.25, y, -0.25), (0.25, y, 0.25), (-0.25, y, 0.25))
    parts.append((light, rng.uniform(0.2, 0.8, 3), 0.0, LAMBERT))
    tris, albedo, rough, mtype = _assemble(parts)
    assert tris.shape[0] == 36, tris.shape
    n_light = light.shape[0]
    emitters = [dict(type=EMITTER_AREA, first_tri=tris.shape[0] - n_light, n_tris=n_light,
                     radiance=(10.0, 10.0, 10.0), position=(0.0, 0.0, 0.0))]
    camera = dict(origin=(0.0, 0.0, 3.5), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_x_deg=40.0)
    return Scene(tris, albedo, rough, mtype, emitters, camera)


CORNELL_FILM = FilmSpec(H=64, W=64, T=256, C=3, start_opl=3.5, bin_width=0.01)


def large_scene(seed: int = SCENE_SEED, hf_res: int = 513, n_spheres: int = 200,
                subdiv_even: int = 4, subdiv_odd: int = 3, size: float = 20.0,
                amplitude: float = 2.0) -> Scene:
    """fBm heightfield (hf_res^2 vertices over size^2 m) plus n_spheres
    icospheres resting on it; 70% Lambertian / 30% GGX conductor materials per
    heightfield patch and per sphere; four 1 m quad lights at 8 m."""
    rng = np.random.default_rng(seed)
    noise = ValueNoise(seed + 1, 2, period=64)
    base_freq = 6.0 / size

    def height(x, z):
        return amplitude * noise.fbm(x * base_freq + 17.0, z * base_freq + 31.0, octaves=5)

    n = hf_res
    xs = np.linspace(-size / 2, size / 2, n)
    X, Z = np.meshgrid(xs, xs, indexing="ij")
    Y = height(X, Z)
    P = np.stack([X, Y, Z], -1)
    a = P[:-1, :-1]
    b = P[1:, :-1]
    c = P[1:, 1:]
    d = P[:-1, 1:]
    # winding with +y normals: (a, d, c) and (a, c, b)
    t1 = np.stack([a, d, c], -2)
    t2 = np.stack([a, c, b], -2)
    hf = np.stack([t1, t2], 2).reshape(-1, 3, 3)
    cells = n - 1
    patch = max(1, cells // 16)
    ci = np.arange(cells)[:, None].repeat(cells, 1)
    cj = np.arange(cells)[None, :].repeat(cells, 0)
    patch_id = ((ci // patch) * (cells // patch + 1) + (cj // patch)).reshape(-1).repeat(2)
    n_patch = int(patch_id.max()) + 1
    p_type = np.where(rng.random(n_patch) < 0.3, GGX, LAMBERT).astype(np.uint32)
    p_alb = np.where(p_type[:, None] == GGX, rng.uniform(0.5, 1.0, (n_patch, 3)), rng.uniform(0.2, 0.8, (n_patch, 3)))
    p_rough = np.where(p_type == GGX, rng.uniform(0.05, 0.5, n_patch), 0.0)
    tris = [hf]
    alb = [p_alb[patch_id]]
    rough = [p_rough[patch_id]]
    mtype = [p_type[patch_id]]
    spheres = {lvl: icosphere(lvl) for lvl in {subdiv_even, subdiv_odd}}
    for k in range(n_spheres):
        r = rng.uniform(0.05, 0.5)
        cx, cz = rng.uniform(-0.45 * size, 0.45 * size, 2)
        cy = float(height(np.array(cx), np.array(cz))) + r
        lvl = subdiv_even if k % 2 == 0 else subdiv_odd
        s = spheres[lvl] * r + np.array([cx, cy, cz])
        if rng.random() < 0.3:
            m, al, ro = GGX, rng.uniform(0.5, 1.0, 3), rng.uniform(0.05, 0.5)
        else:
            m, al, ro = LAMBERT, rng.uniform(0.2, 0.8, 3), 0.0
        tris.append(s)
        alb.append(np.broadcast_to(al, (len(s), 3)))
        rough.append(np.full(len(s), ro))
        mtype.append(np.full(len(s), m, np.uint32))
    emitters = []
    n_before = sum(len(t) for t in tris)
    for (lx, lz) in ((-4.0, -4.0), (4.0, -4.0), (-4.0, 4.0), (4.0, 4.0)):
        y = 8.0
        q = quad((lx - 0.5, y, lz + 0.5), (lx + 0.5, y, lz + 0.5), (lx + 0.5, y, lz - 0.5), (lx - 0.5, y, lz - 0.5))
        # normal must face down (-y)
        nrm = np.cross(q[0, 1] - q[0, 0], q[0, 2] - q[0, 0])
        if nrm[1] > 0:
            q = q[:, ::-1, :]
        emitters.append(dict(type=EMITTER_AREA, first_tri=n_before, n_tris=2,
                             radiance=(20.0, 20.0, 20.0), position=(0.0, 0.0, 0.0)))
        n_before += 2
        tris.append(q)
        alb.append(np.full((2, 3), 0.5))
        rough.append(np.zeros(2))
        mtype.append(np.zeros(2, np.uint32))
    tris = np.concatenate(tris).astype(np.float32)
    albedo = np.ascontiguousarray(np.concatenate(alb), np.float32)
    rough = np.concatenate(rough).astype(np.float32)
    mtype = np.concatenate(mtype).astype(np.uint32)
    a30 = math.radians(30.0)
    origin = (0.0, 6.0, 12.0)
    target = (0.0, 6.0 - math.sin(a30), 12.0 - math.cos(a30))
    camera = dict(origin=origin, target=target, up=(0.0, 1.0, 0.0), fov_x_deg=50.0)
    return Scene(tris, albedo, rough, mtype, emitters, camera)


LARGE_FILM = FilmSpec(H=512, W=512, T=2048, C=3, start_opl=12.0, bin_width=0.005)


def diff_scene(seed: int = SCENE_SEED) -> Scene:
    """The large scene cut to ~97k triangles (129^2 heightfield, level-2 spheres)."""
    return large_scene(seed, hf_res=129, n_spheres=200, subdiv_even=2, subdiv_odd=2)


DIFF_FILM = FilmSpec(H=256, W=256, T=512, C=3, start_opl=15.0, bin_width=0.005)


def perturbed_albedo(scene: Scene, seed: int = TARGET_SEED, amount: float = 0.2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    f = rng.uniform(1.0 - amount, 1.0 + amount, (scene.n_tris, 1))
    return np.ascontiguousarray(np.clip(scene.albedo * f, 0.0, 1.0), np.float32)


def nlos_scene(seed: int = SCENE_SEED) -> Scene:
    """1x1 m relay wall at z=0 facing +z (albedo 0.8) and a hidden ~49k-triangle
    mesh 0.54-1.52 m in front of it: two bumpy level-5 icospheres and an extruded
    8-point star."""
    rng = np.random.default_rng(seed)
    wall = quad((-0.5, -0.5, 0.0), (0.5, -0.5, 0.0), (0.5, 0.5, 0.0), (-0.5, 0.5, 0.0))
    noise3 = ValueNoise(seed + 7, 3, period=32)
    parts = [wall]
    centers = [(-0.2, 0.1, 0.8), (0.25, -0.15, 1.25)]
    base = icosphere(5)
    for k, c in enumerate(centers):
        dirs = base.reshape(-1, 3)
        bump = noise3(dirs[:, 0] * 4 + 5 * k, dirs[:, 1] * 4 + 3, dirs[:, 2] * 4 + 11)
        r = 0.25 + 0.02 * (2.0 * bump - 1.0)
        s = (dirs * r[:, None]).reshape(-1, 3, 3) + np.array(c)
        parts.append(s)
    # extruded 8-point star: 128 outline vertices x 32 rings, fan caps
    n_out, n_ring, depth = 128, 32, 0.1
    ang = np.arange(n_out) * 2 * math.pi / n_out
    spikes = 8
    rad = 0.12 + 0.08 * (0.5 + 0.5 * np.cos(ang * spikes))
    ox, oy = rad * np.cos(ang), rad * np.sin(ang)
    sc = np.array([0.05, 0.25, 1.0])
    rings = [np.stack([ox, oy, np.full(n_out, z)], -1) + sc for z in np.linspace(-depth / 2, depth / 2, n_ring + 1)]
    side = []
    for r in range(n_ring):
        A, B = rings[r], rings[r + 1]
        for i in range(n_out):
            j = (i + 1) % n_out
            side.append(quad(A[i], A[j], B[j], B[i]))
    side = np.concatenate(side)
    cap0 = np.stack([np.broadcast_to(sc + [0, 0, -depth / 2], (n_out, 3)), rings[0][(np.arange(n_out) + 1) % n_out], rings[0]], 1)
    cap1 = np.stack([np.broadcast_to(sc + [0, 0, depth / 2], (n_out, 3)), rings[-1], rings[-1][(np.arange(n_out) + 1) % n_out]], 1)
    parts += [side, cap0, cap1]
    tris = np.concatenate(parts).astype(np.float32)
    n = tris.shape[0]
    albedo = np.full((n, 3), 0.8, np.float32)
    rough = np.zeros(n, np.float32)
    mtype = np.zeros(n, np.uint32)
    camera = dict(origin=(0.0, 0.0, 2.0), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fov_x_deg=40.0)
    wall_info = dict(center=(0.0, 0.0, 0.0), size=1.0, normal=(0.0, 0.0, 1.0), albedo=0.8)
    return Scene(tris, albedo, rough, mtype, [], camera, hidden=(2, n - 2), wall=wall_info)


def wall_grid(nx: int, ny: int, size: float = 1.0, z: float = 0.0) -> np.ndarray:
    """Cell-centred nx*ny grid of points on the relay wall, row-major (y, x)."""
    xs = (np.arange(nx) + 0.5) / nx * size - size / 2
    ys = (np.arange(ny) + 0.5) / ny * size - size / 2
    Yg, Xg = np.meshgrid(ys, xs, indexing="ij")
    return np.ascontiguousarray(np.stack([Xg, Yg, np.full_like(Xg, z)], -1).reshape(-1, 3), np.float32)


NLOS_T, NLOS_W, NLOS_START = 4096, 0.003, 0.0


def media_scene(seed: int = SCENE_SEED, res: int = 128) -> Scene:
    """The Cornell box filled with a res^3 heterogeneous medium, sigma_t in
    [0.1, 2] /m from seeded 3-D fBm, single-scatter albedo 0.9, HG g = 0.3."""
    s = cornell_box(seed)
    noise3 = ValueNoise(seed + 3, 3, period=32)
    c = (np.arange(res) + 0.5) / res * 8.0
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    f = noise3.fbm(X, Y, Z, octaves=4)
    f = (f - f.min()) / (f.max() - f.min())
    dens = (0.1 + 1.9 * f).astype(np.float32)   # [z][y][x]
    s.medium = dict(lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), density=np.ascontiguousarray(dens),
                    albedo=0.9, g=0.3)
    return s


MEDIA_FILM = FilmSpec(H=256, W=256, T=1024, C=3, start_opl=3.5, bin_width=0.005)


def homogeneous_medium(sigma: float, res: int = 4, albedo: float = 0.9, g: float = 0.3,
                       lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0)) -> dict:
    return dict(lo=lo, hi=hi, density=np.full((res, res, res), sigma, np.float32), albedo=albedo, g=g)


# ----------------------------------------------------------------------------
# closed-form test scenes
# ----------------------------------------------------------------------------

def point_light_plane(albedo: float = 0.6, intensity: float = 5.0, light_pos=(0.3, 1.2, -0.2),
                      cam_height: float = 2.0, fov: float = 50.0) -> Scene:
    """Lambertian plane y=0 (20x20 m) lit by one point emitter, camera above."""
    S = 10.0
    plane = quad((-S, 0.0, S), (S, 0.0, S), (S, 0.0, -S), (-S, 0.0, -S))
    if np.cross(plane[0, 1] - plane[0, 0], plane[0, 2] - plane[0, 0])[1] < 0:
        plane = plane[:, ::-1, :]
    tris = plane.astype(np.float32)
    albedo = np.full((2, 3), albedo, np.float32)
    emitters = [dict(type=EMITTER_POINT, first_tri=0, n_tris=0, radiance=(intensity,) * 3, position=tuple(light_pos))]
    camera = dict(origin=(0.0, cam_height, 0.5), target=(0.0, 0.0, -0.3), up=(0.0, 1.0, 0.0), fov_x_deg=fov)
    return Scene(tris, albedo, np.zeros(2, np.float32), np.zeros(2, np.uint32), emitters, camera)


def mirror_wall(f0=(0.9, 0.6, 0.3), rough: float = 1e-4, wall_albedo: float = 0.7) -> Scene:
    """A near-perfect conductor floor (y = 0, GGX) reflecting a Lambertian wall
    (z = -3) lit by a point emitter off to the side; the camera looks down at
    the floor, so most pixels see the wall through one specular reflection."""
    S = 10.0
    floor = quad((-S, 0.0, S), (S, 0.0, S), (S, 0.0, -S), (-S, 0.0, -S))
    wall = quad((-S, 0.0, -3.0), (S, 0.0, -3.0), (S, 2 * S, -3.0), (-S, 2 * S, -3.0))
    tris = np.concatenate([floor, wall]).astype(np.float32)
    albedo = np.concatenate([np.tile(np.array(f0, np.float32), (2, 1)), np.full((2, 3), wall_albedo, np.float32)])
    rough_a = np.array([rough, rough, 0.0, 0.0], np.float32)
    mtype = np.array([1, 1, 0, 0], np.uint32)
    emitters = [dict(type=EMITTER_POINT, first_tri=0, n_tris=0, radiance=(8.0,) * 3, position=(2.5, 1.5, -2.0))]
    camera = dict(origin=(0.0, 2.0, 2.0), target=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0), fov_x_deg=40.0)
    return Scene(tris, albedo, rough_a, mtype, emitters, camera)


def mirror_corner(f0_floor=(0.9, 0.6, 0.3), f0_wall=(0.5, 0.8, 0.95), rough: float = 1e-4) -> Scene:
    """Two near-perfect conductors, the floor (y = 0) and a back wall (z = -3),
    and a Lambertian ceiling (y = 6) lit by a point emitter off to the side:
    the camera sees the ceiling through a reflection in the floor followed by
    one in the back wall."""
    S = 12.0
    floor = quad((-S, 0.0, S), (S, 0.0, S), (S, 0.0, -3.0), (-S, 0.0, -3.0))
    wall = quad((-S, 0.0, -3.0), (S, 0.0, -3.0), (S, 6.0, -3.0), (-S, 6.0, -3.0))
    ceil = quad((-S, 6.0, -3.0), (S, 6.0, -3.0), (S, 6.0, S), (-S, 6.0, S))
    tris = np.concatenate([floor, wall, ceil]).astype(np.float32)
    albedo = np.concatenate([np.tile(np.array(f0_floor, np.float32), (2, 1)),
                             np.tile(np.array(f0_wall, np.float32), (2, 1)), np.full((2, 3), 0.7, np.float32)])
    rough_a = np.array([rough, rough, rough, rough, 0.0, 0.0], np.float32)
    mtype = np.array([1, 1, 1, 1, 0, 0], np.uint32)
    emitters = [dict(type=EMITTER_POINT, first_tri=0, n_tris=0, radiance=(30.0,) * 3, position=(6.0, 5.5, 2.0))]
    camera = dict(origin=(0.0, 2.0, 2.0), target=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0), fov_x_deg=40.0)
    return Scene(tris, albedo, rough_a, mtype, emitters, camera)


def furnace_sphere(level: int = 4, radius: float = 1.0, albedo: float = 0.5, radiance: float = 1.0) -> Scene:
    """Closed inward-facing icosphere, every triangle emissive and Lambertian;
    the camera sits at the centre."""
    s = icosphere(level)[:, ::-1, :] * radius      # flip winding: normals inward
    tris = np.ascontiguousarray(s, np.float32)
    n = tris.shape[0]
    emitters = [dict(type=EMITTER_AREA, first_tri=0, n_tris=n, radiance=(radiance,) * 3, position=(0.0, 0.0, 0.0))]
    camera = dict(origin=(0.0, 0.0, 0.0), target=(0.0, 0.0, -1.0), up=(0.0, 1.0, 0.0), fov_x_deg=60.0)
    return Scene(tris, np.full((n, 3), albedo, np.float32), np.zeros(n, np.float32), np.zeros(n, np.uint32), emitters, camera)


def random_mesh(seed: int, n_tris: int, extent: float = 1.0) -> np.ndarray:
    """Random small triangles in [-extent, extent]^3 for intersection tests."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-extent, extent, (n_tris, 1, 3))
    e = rng.normal(0.0, 0.25 * extent, (n_tris, 3, 3))
    return (c + e).astype(np.float32)


def random_rays(seed: int, n: int, extent: float = 1.0):
    rng = np.random.default_rng(seed)
    o = rng.uniform(-2 * extent, 2 * extent, (n, 3))
    tgt = rng.uniform(-extent, extent, (n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o.astype(np.float32), d.astype(np.float32)
