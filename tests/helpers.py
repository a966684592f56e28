"""Small shared builders for tests: hand-made cameras, meshes and worlds."""
from __future__ import annotations

import numpy as np

from paper_1510_05613_gb300 import synth


def top_down_camera(W: int, H: int, f: float, cx: float, cy: float, height: float = 2.0) -> synth.Camera:
    """Camera at (0, 0, height) looking straight down: x_c = x_w, y_c = -y_w,
    z_c = height - z_w (all exact in binary32 for dyadic inputs)."""
    T = np.array([[1, 0, 0, 0], [0, -1, 0, 0], [0, 0, -1, height]], np.float32)
    return synth.Camera(W, H, f, f, cx, cy, T)


def identity_grid() -> synth.PoseGrid:
    """A single pose: x = y = 0, yaw 0 (cos 1, sin 0)."""
    return synth.PoseGrid(np.zeros(1, np.float32), np.zeros(1, np.float32), np.array([[1.0, 0.0]], np.float32))


def tri_mesh(verts, name="tri", vol=(0.0, 1.0, -1.0)) -> synth.Mesh:
    """One-triangle mesh (object frame); V(O) empty by default."""
    v = np.asarray(verts, np.float32).reshape(3, 3)
    return synth.Mesh(name, v, np.array([[0, 1, 2]], np.int32), vol[0], vol[1], vol[2])


def signed_area2(a, b, c):
    """Twice the signed area of triangle abc in a y-down pixel frame, written
    as the textbook cross product (b - a) x (c - a) with y negated, so that
    a triangle seen counter-clockwise by a y-up viewer is positive."""
    ax, ay = a
    bx, by = b
    cx, cy = c
    return -((bx - ax) * (cy - ay) - (by - ay) * (cx - ax))
