"""Seeded synthetic inputs for the tetrahedron rasterizer.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds only input generation: structured tetrahedral grids,
scalar fields sampled at the grid vertices, per-vertex colours, pinhole
cameras and upstream image gradients.  None of the rendering method's
arithmetic (opacity, projection for binning, blending, gradients) lives here.

Conventions
-----------
* Grid: ``n`` cubes per axis spanning [-1, 1]^3, vertex ``(i, j, k)`` has index
  ``i + (n+1) * (j + (n+1) * k)``; each cube is split into 6 tetrahedra by the
  Kuhn (Freudenthal) rule: for every permutation ``pi`` of the axes in
  lexicographic order the tet is ``(v0, v0+e_pi0, v0+e_pi0+e_pi1, v0+(1,1,1))``.
  This split is conforming across cubes.  Tets are ordered cube-major (i
  fastest), permutation-minor.  The paper's structured grids (Sec. 3.1, App. B)
  follow DMTet; the split rule is not stated there.
* Camera: world->camera rotation ``R`` (row-major) and translation ``t`` with
  OpenCV axes (x right, y down, z forward), pinhole intrinsics
  ``fx = fy = W / (2 tan(fov/2))``, ``cx = W/2``, ``cy = H/2``; pixel ``(i, j)``
  has its centre at ``(i + 0.5, j + 0.5)``.
* Random numbers: ``numpy.random.default_rng(seed)``.
"""

from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

FOV_DEG = 49.0
ZNEAR = 0.1
CAM_RADIUS = 2.5

# ----------------------------------------------------------------------------
# grids
# ----------------------------------------------------------------------------

_PERMS = list(itertools.permutations(range(3)))  # lexicographic order


def grid_vertices(n: int) -> np.ndarray:
    """(n+1)^3 x 3 float32 vertex positions on [-1,1]^3, i fastest."""
    ax = (-1.0 + 2.0 * np.arange(n + 1, dtype=np.float64) / n)
    k, j, i = np.meshgrid(ax, ax, ax, indexing="ij")
    V = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    return V.astype(np.float32)


def grid_tets(n: int) -> np.ndarray:
    """6 n^3 x 4 int32 tet indices (Kuhn split), cube-major, permutation-minor."""
    m = n + 1
    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # cube order: i fastest
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    v0 = ci + m * (cj + m * ck)
    step = np.array([1, m, m * m], dtype=np.int64)
    out = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for p, perm in enumerate(_PERMS):
        a = v0
        b = a + step[perm[0]]
        c = b + step[perm[1]]
        d = c + step[perm[2]]
        out[:, p, 0] = a
        out[:, p, 1] = b
        out[:, p, 2] = c
        out[:, p, 3] = d
    return out.reshape(-1, 4).astype(np.int32)


# ----------------------------------------------------------------------------
# fields sampled at vertices
# ----------------------------------------------------------------------------

def sdf_sphere(V: np.ndarray, radius: float = 0.5, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    x = V.astype(np.float64) - np.asarray(center, dtype=np.float64)
    return np.linalg.norm(x, axis=1) - radius


def sdf_torus(V: np.ndarray, R: float = 0.5, r: float = 0.2) -> np.ndarray:
    """Torus about the z axis."""
    x = V.astype(np.float64)
    q = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2) - R
    return np.sqrt(q * q + x[:, 2] ** 2) - r


def sdf_spheres_union(V: np.ndarray, centers: np.ndarray, radii: np.ndarray) -> np.ndarray:
    x = V.astype(np.float64)
    d = [np.linalg.norm(x - c, axis=1) - r for c, r in zip(centers, radii)]
    return np.min(np.stack(d, 0), axis=0)


def value_noise(V: np.ndarray, rng: np.random.Generator, freqs=(4, 8, 16),
                amps=(0.02, 0.01, 0.005)) -> np.ndarray:
    """Multi-octave value noise on [-1,1]^3: a lattice of U[-1,1] values with
    ``freq`` cells across [-1,1], smoothstep-weighted trilinear interpolation."""
    x = V.astype(np.float64)
    out = np.zeros(len(x))
    for fq, amp in zip(freqs, amps):
        lat = rng.uniform(-1.0, 1.0, size=(fq + 1, fq + 1, fq + 1))
        g = (x + 1.0) * 0.5 * fq
        i0 = np.clip(np.floor(g).astype(np.int64), 0, fq - 1)
        w = g - i0
        w = w * w * (3.0 - 2.0 * w)
        acc = np.zeros(len(x))
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    wt = ((w[:, 0] if dx else 1 - w[:, 0]) *
                          (w[:, 1] if dy else 1 - w[:, 1]) *
                          (w[:, 2] if dz else 1 - w[:, 2]))
                    acc += wt * lat[i0[:, 0] + dx, i0[:, 1] + dy, i0[:, 2] + dz]
        out += amp * acc
    return out


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Camera:
    R: np.ndarray          # 3x3 float32, world -> camera, row-major
    t: np.ndarray          # 3 float32
    fx: float
    fy: float
    cx: float
    cy: float
    znear: float
    width: int
    height: int

    def astuple(self):
        return (self.R, self.t, self.fx, self.fy, self.cx, self.cy, self.znear,
                self.width, self.height)


def look_at_camera(pos, width: int, height: int, fov_deg: float = FOV_DEG,
                   znear: float = ZNEAR, target=(0.0, 0.0, 0.0)) -> Camera:
    """Pinhole camera at ``pos`` looking at ``target`` with up hint +z (+y when
    the view direction is collinear with z).  All maths in float64, stored as
    float32."""
    c = np.asarray(pos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - c
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 0.0, 1.0])
    if abs(np.dot(fwd, up)) > 0.999:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], 0)
    t = -R @ c
    fx = width / (2.0 * math.tan(math.radians(fov_deg) * 0.5))
    return Camera(R=R.astype(np.float32), t=t.astype(np.float32), fx=float(np.float32(fx)),
                  fy=float(np.float32(fx)), cx=float(np.float32(width * 0.5)),
                  cy=float(np.float32(height * 0.5)), znear=float(np.float32(znear)),
                  width=int(width), height=int(height))


def orbit_camera(azim_deg: float, elev_deg: float, width: int, height: int,
                 radius: float = CAM_RADIUS) -> Camera:
    a, e = math.radians(azim_deg), math.radians(elev_deg)
    pos = radius * np.array([math.cos(e) * math.cos(a), math.cos(e) * math.sin(a), math.sin(e)])
    return look_at_camera(pos, width, height)


def random_camera(rng: np.random.Generator, width: int, height: int,
                  radius: float = CAM_RADIUS) -> Camera:
    """Uniform on the sphere of ``radius`` (normalised Gaussian)."""
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    return look_at_camera(radius * d, width, height)


# ----------------------------------------------------------------------------
# scenes (the workloads)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Scene:
    n: int
    V: np.ndarray      # N x 3 float32
    T: np.ndarray      # K x 4 int32
    f: np.ndarray      # N float32
    rgb: np.ndarray    # N x 3 float32
    cams: list
    name: str = ""

    @property
    def N(self):
        return len(self.V)

    @property
    def K(self):
        return len(self.T)


def scene_sphere16(res: int = 128) -> Scene:
    """16^3 cubes (24,576 tets, 4,913 vertices); sphere SDF |x|-0.5 plus
    N(0, 0.01^2); rgb U[0,1]; one camera at radius 2.5, azimuth 30 deg,
    elevation 20 deg; 128x128; seed 0."""
    rng = np.random.default_rng(0)
    n = 16
    V = grid_vertices(n)
    T = grid_tets(n)
    f = (sdf_sphere(V) + rng.normal(0.0, 0.01, size=len(V))).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, size=(len(V), 3)).astype(np.float32)
    cams = [orbit_camera(30.0, 20.0, res, res)]
    return Scene(n, V, T, f, rgb, cams, "sphere16")


def scene_torus64(res: int = 512) -> Scene:
    """64^3 cubes (1,572,864 tets, 274,625 vertices); torus (R=0.5, r=0.2) SDF
    plus 3-octave value noise (amplitudes 0.02, 0.01, 0.005 at 4, 8, 16 cells);
    rgb U[0,1]; one random camera on the radius-2.5 sphere; 512x512; seed 1."""
    rng = np.random.default_rng(1)
    n = 64
    V = grid_vertices(n)
    T = grid_tets(n)
    f = (sdf_torus(V) + value_noise(V, rng)).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, size=(len(V), 3)).astype(np.float32)
    cams = [random_camera(rng, res, res)]
    return Scene(n, V, T, f, rgb, cams, "torus64")


def spheres3_field(V: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    centers = rng.uniform(-0.4, 0.4, size=(3, 3))
    radii = rng.uniform(0.2, 0.4, size=3)
    return sdf_spheres_union(V, centers, radii)


def scene_spheres128(res: int = 512, n_views: int = 4, n: int = 128,
                     tets: bool = True) -> Scene:
    """128^3 cubes (12,582,912 tets, 2,146,689 vertices); union of 3 random
    spheres (centres U[-0.4,0.4]^3, radii U[0.2,0.4]) plus N(0, 0.01^2); rgb
    U[0,1]; 4 random views at 512x512; seed 2.  ``tets=False`` leaves the tet
    array empty (for callers that only need a sub-grid)."""
    rng = np.random.default_rng(2)
    V = grid_vertices(n)
    T = grid_tets(n) if tets else np.zeros((0, 4), np.int32)
    f = (spheres3_field(V, rng) + rng.normal(0.0, 0.01, size=len(V))).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, size=(len(V), 3)).astype(np.float32)
    cams = [random_camera(rng, res, res) for _ in range(n_views)]
    return Scene(n, V, T, f, rgb, cams, "spheres128")


def subgrid(scene: Scene, lo: int, hi: int) -> Scene:
    """Cubes [lo, hi)^3 of a structured grid scene as a standalone grid
    (vertices re-indexed, same positions, fields and cameras)."""
    n, m = scene.n, scene.n + 1
    ns = hi - lo
    idx = np.arange(lo, hi + 1)
    kk, jj, ii = np.meshgrid(idx, idx, idx, indexing="ij")
    old = (ii + m * (jj + m * kk)).ravel()
    V = scene.V[old]
    T = grid_tets(ns)
    return Scene(ns, V, T, scene.f[old], scene.rgb[old], list(scene.cams),
                 f"{scene.name}[{lo}:{hi}]")


def upstream_grads(seed: int, cams) -> list:
    """dL/d{image, alpha, depth} ~ N(0,1) per view, from default_rng(seed+1000)."""
    rng = np.random.default_rng(seed + 1000)
    out = []
    for c in cams:
        H, W = c.height, c.width
        gi = rng.normal(size=(3, H, W)).astype(np.float32)
        ga = rng.normal(size=(H, W)).astype(np.float32)
        gd = rng.normal(size=(H, W)).astype(np.float32)
        out.append((gi, ga, gd))
    return out


_TOPOLOGY: dict = {}


def shared_grid(n: int) -> tuple:
    """(V, T) of the n^3 grid, built once per n and shared by every caller
    (the batched and served workloads hold many scenes of a few
    resolutions).  The arrays must not be modified."""
    if n not in _TOPOLOGY:
        _TOPOLOGY[n] = (grid_vertices(n), grid_tets(n))
    return _TOPOLOGY[n]


def random_scene(rng: np.random.Generator, n: int, kind: str = "sphere",
                 noise: float = 0.01) -> tuple:
    """Vertex fields for a batched/served scene: a random sphere or torus SDF
    plus N(0, noise^2); rgb U[0,1].  V and T are the shared grid of
    ``shared_grid(n)`` (do not modify them)."""
    V, T = shared_grid(n)
    if kind == "sphere":
        c = rng.uniform(-0.2, 0.2, size=3)
        r = rng.uniform(0.3, 0.6)
        f = sdf_sphere(V, r, c)
    else:
        f = sdf_torus(V, rng.uniform(0.4, 0.6), rng.uniform(0.15, 0.25))
    f = (f + rng.normal(0.0, noise, size=len(V))).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, size=(len(V), 3)).astype(np.float32)
    return V, T, f, rgb


S_HEADLINE = 175.0
