"""Pinhole cameras in the library's convention: world -> camera x_c = R v + t
with OpenCV axes (x right, y down, z forward), pixel (i, j) centred at
(i + 0.5, j + 0.5)."""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Camera:
    R: np.ndarray          # 3x3 float32, row-major world -> camera
    t: np.ndarray          # 3 float32
    fx: float
    fy: float
    cx: float
    cy: float
    znear: float
    width: int
    height: int


def look_at(pos, width: int, height: int, fov_deg: float = 49.0, znear: float = 0.1,
            target=(0.0, 0.0, 0.0)) -> Camera:
    """Camera at ``pos`` looking at ``target``, up hint +z (+y when looking
    along z); horizontal field of view ``fov_deg``."""
    c = np.asarray(pos, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - c
    fwd /= np.linalg.norm(fwd)
    up = np.array([0.0, 0.0, 1.0])
    if abs(float(np.dot(fwd, up))) > 0.999:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], 0)
    t = -R @ c
    f = width / (2.0 * math.tan(math.radians(fov_deg) * 0.5))
    return Camera(R.astype(np.float32), t.astype(np.float32), float(np.float32(f)),
                  float(np.float32(f)), float(np.float32(width * 0.5)),
                  float(np.float32(height * 0.5)), float(np.float32(znear)), int(width),
                  int(height))


def on_sphere(rng: np.random.Generator, width: int, height: int, radius: float = 2.5) -> Camera:
    """Uniformly random position on a sphere around the origin, looking at it."""
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    return look_at(radius * d, width, height)


def orbit(azim_deg: float, elev_deg: float, width: int, height: int,
          radius: float = 2.5) -> Camera:
    a, e = math.radians(azim_deg), math.radians(elev_deg)
    return look_at(radius * np.array([math.cos(e) * math.cos(a), math.cos(e) * math.sin(a),
                                      math.sin(e)]), width, height)
