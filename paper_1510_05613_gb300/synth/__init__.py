"""Seeded synthetic PERCH workloads: procedural meshes, pose grids, camera,
ground-truth scenes and simulated noisy depth observations.

This module is input generation only. It holds none of the method's
arithmetic (no z-buffer rendering, no explanation cost, no search): both the
CPU oracle and the CUDA library consume what it produces. The observation is
made by a double-precision ray caster (``sensor.c``), a different algorithm
from the fixed-point rasteriser the method uses.

The paper's own data (the occlusion dataset of its Sec. V-A, 36 CAD models)
is not available, so procedural tabletop objects with the shapes and sizes of
the workloads below stand in for it. The problem statement (Sec. III) fixes the
structure: known object models, known object count and types, 3-DoF poses
(x, y, yaw) on a table, a known sensor pose and intrinsics, and an observed
cloud containing only object points.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SENSOR_SRC = os.path.join(_HERE, "sensor.c")
_SENSOR_LIB = os.path.join(_HERE, "libperch_sensor.so")

# ---------------------------------------------------------------------------
# counter-based random numbers (SplitMix64, Steele/Lea/Flood 2014)
# ---------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Values ``offset .. offset+n-1`` of the SplitMix64 stream of ``seed``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller over two interleaved uniform streams."""
    u = uniform(seed, 2 * n)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def substream(seed: int, tag: int) -> int:
    """Independent seed for a named sub-stream of a scene's seed."""
    return int(splitmix64(seed * 7919 + tag, 1)[0])


# ---------------------------------------------------------------------------
# procedural meshes (object frame: z up, base on z = 0, CCW seen from outside)
# ---------------------------------------------------------------------------
@dataclass
class Mesh:
    name: str
    verts: np.ndarray  # float32 (V, 3)
    tris: np.ndarray  # int32 (T, 3)
    vol_r: float  # V(O): inscribed vertical cylinder about the object origin
    vol_zlo: float
    vol_zhi: float
    # the closed-form solid the mesh describes, when it has one (see Volume)
    volume: "Volume | None" = None
    # rotational symmetry order about the vertical axis: turning the mesh by
    # 2 pi / sym maps its vertex set onto itself (1 = none)
    sym: int = 1

    @property
    def n_verts(self) -> int:
        return int(self.verts.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def footprint_radius(self) -> float:
        v = self.verts.astype(np.float64)
        return float(np.sqrt((v[:, 0] ** 2 + v[:, 1] ** 2).max()))


# closed-form object volumes V(O) (Sec. III-A: the volume the object
# occupies, in closed form where there is one)
VOL_CYLINDER, VOL_BOX, VOL_PRISM, VOL_SUPERQUADRIC = 0, 1, 2, 3


@dataclass
class Volume:
    """Closed-form solid of one mesh, in its object frame (z up, base on
    z = 0). kind VOL_BOX: |x| <= p[0], |y| <= p[1], zlo <= z <= zhi.
    VOL_PRISM: the regular n-gon whose vertex k is at angle 2 pi k / n and
    radius p[0] (apothem p[1]): every face k has n_k . (x, y) <= p[1] with the
    outward unit normals n_k = normals[k] (angle (2k + 1) pi / n), and
    zlo <= z <= zhi. VOL_SUPERQUADRIC with exponent pair n: semi-axes p[0..2],
    centre height p[3]; X = x / p[0], Y = y / p[1], Z = (z - p[3]) / p[2];
    n = 1 (eps1 = eps2 = 1, ellipsoid): X^2 + Y^2 + Z^2 <= 1; n = 2
    (eps1 = 0.5, eps2 = 1): (X^2 + Y^2)^2 + Z^4 <= 1. The parameters are
    binary32 as given to the oracle and the library, computed here in
    double; the normals are the input data both sides use."""
    kind: int
    n: int
    p: np.ndarray  # float32 (4,)
    zlo: float
    zhi: float
    normals: np.ndarray  # float32 (n, 2) for VOL_PRISM, else (0, 2)


def box_volume(a: float, b: float, h: float) -> Volume:
    return Volume(VOL_BOX, 0, np.array([a / 2, b / 2, 0, 0], np.float32), 0.0, float(np.float32(h)),
                  np.zeros((0, 2), np.float32))


def prism_volume(R: float, n: int, h: float) -> Volume:
    ang = [(2 * k + 1) * math.pi / n for k in range(n)]
    normals = np.array([[math.cos(t), math.sin(t)] for t in ang], np.float64).astype(np.float32)
    p = np.array([R, R * math.cos(math.pi / n), 0, 0], np.float64).astype(np.float32)
    return Volume(VOL_PRISM, n, p, 0.0, float(np.float32(h)), normals)


def superquadric_volume(a1: float, a2: float, a3: float, e1: float, e2: float) -> "Volume | None":
    n = {(1.0, 1.0): 1, (0.5, 1.0): 2}.get((float(e1), float(e2)))
    if n is None:
        return None  # exponents without a polynomial closed form here: the inscribed cylinder stays
    p = np.array([a1, a2, a3, a3], np.float32)
    return Volume(VOL_SUPERQUADRIC, n, p, float(np.float32(0.0)), float(np.float32(2 * a3)),
                  np.zeros((0, 2), np.float32))


def _orient_outward(verts: np.ndarray, tris: np.ndarray, centre) -> np.ndarray:
    """Make every triangle's normal point away from ``centre`` (valid for
    star-shaped, here convex, solids)."""
    v = verts.astype(np.float64)
    a, b, c = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    n = np.cross(b - a, c - a)
    out = ((a + b + c) / 3.0) - np.asarray(centre, np.float64)
    flip = (n * out).sum(1) < 0
    t = tris.copy()
    t[flip, 1], t[flip, 2] = tris[flip, 2], tris[flip, 1]
    return t


def _weld(points: np.ndarray, tris: np.ndarray, decimals: int = 9):
    key = np.round(points, decimals)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    inv = inv.reshape(-1)
    new_pts = points[first]
    new_tris = inv[tris]
    keep = (new_tris[:, 0] != new_tris[:, 1]) & (new_tris[:, 1] != new_tris[:, 2]) & (new_tris[:, 0] != new_tris[:, 2])
    return new_pts, new_tris[keep]


def box_mesh(a: float, b: float, h: float, n: int, name: str = "box") -> Mesh:
    """Box of size a x b x h (x, y, z), every face split into n x n quads."""
    pts, tris = [], []
    size = np.array([a, b, h])
    lo = np.array([-a / 2, -b / 2, 0.0])
    # (normal axis, sign, u axis, v axis) with u x v = sign * normal
    faces = [(2, 1, 0, 1), (2, -1, 1, 0), (0, 1, 1, 2), (0, -1, 2, 1), (1, 1, 2, 0), (1, -1, 0, 2)]
    for ax, sg, ua, va in faces:
        base = len(pts)
        for j in range(n + 1):
            for i in range(n + 1):
                p = np.zeros(3)
                p[ax] = 1.0 if sg > 0 else 0.0
                p[ua] = i / n
                p[va] = j / n
                pts.append(lo + p * size)
        for j in range(n):
            for i in range(n):
                q00 = base + j * (n + 1) + i
                q10, q01, q11 = q00 + 1, q00 + n + 1, q00 + n + 2
                tris.append((q00, q10, q11))
                tris.append((q00, q11, q01))
    P, T = _weld(np.array(pts), np.array(tris, np.int64))
    T = _orient_outward(P, T, (0.0, 0.0, h / 2))
    r = 0.9 * min(a, b) / 2
    return Mesh(name, P.astype(np.float32), T.astype(np.int32), r, 0.05 * h, 0.95 * h, box_volume(a, b, h),
                4 if a == b else 2)


def cylinder_mesh(R: float, h: float, n_seg: int, n_rings: int, name: str = "cylinder") -> Mesh:
    """Closed n-gon cylinder: side split into n_rings bands, fan caps."""
    pts = []
    for l in range(n_rings + 1):
        z = h * l / n_rings
        for k in range(n_seg):
            phi = 2.0 * math.pi * k / n_seg
            pts.append((R * math.cos(phi), R * math.sin(phi), z))
    top_c = len(pts); pts.append((0.0, 0.0, h))
    bot_c = len(pts); pts.append((0.0, 0.0, 0.0))
    tris = []
    for l in range(n_rings):
        for k in range(n_seg):
            a = l * n_seg + k
            b = l * n_seg + (k + 1) % n_seg
            c = (l + 1) * n_seg + (k + 1) % n_seg
            d = (l + 1) * n_seg + k
            tris.append((a, b, c)); tris.append((a, c, d))
    for k in range(n_seg):
        tris.append((top_c, n_rings * n_seg + k, n_rings * n_seg + (k + 1) % n_seg))
        tris.append((bot_c, (k + 1) % n_seg, k))
    P, T = np.array(pts), np.array(tris, np.int64)
    T = _orient_outward(P, T, (0.0, 0.0, h / 2))
    r = 0.9 * R * math.cos(math.pi / n_seg)
    return Mesh(name, P.astype(np.float32), T.astype(np.int32), r, 0.05 * h, 0.95 * h, prism_volume(R, n_seg, h),
                n_seg)


def _spow(x, e):
    return np.sign(x) * np.abs(x) ** e


def superquadric_mesh(a1: float, a2: float, a3: float, e1: float, e2: float,
                      n_eta: int, n_omega: int, name: str = "superquadric") -> Mesh:
    """Superquadric x = a1 C(eta)^e1 C(w)^e2, y = a2 C(eta)^e1 S(w)^e2,
    z = a3 S(eta)^e1 (signed powers), shifted so its base sits on z = 0."""
    etas = np.linspace(-math.pi / 2, math.pi / 2, n_eta + 1)[1:-1]
    oms = np.linspace(-math.pi, math.pi, n_omega, endpoint=False)
    E, O = np.meshgrid(etas, oms, indexing="ij")
    x = a1 * _spow(np.cos(E), e1) * _spow(np.cos(O), e2)
    y = a2 * _spow(np.cos(E), e1) * _spow(np.sin(O), e2)
    z = a3 * _spow(np.sin(E), e1) + a3
    pts = list(np.stack([x, y, z], -1).reshape(-1, 3))
    nr = len(etas)
    bot = len(pts); pts.append((0.0, 0.0, 0.0))
    top = len(pts); pts.append((0.0, 0.0, 2 * a3))
    tris = []
    for l in range(nr - 1):
        for k in range(n_omega):
            a = l * n_omega + k
            b = l * n_omega + (k + 1) % n_omega
            c = (l + 1) * n_omega + (k + 1) % n_omega
            d = (l + 1) * n_omega + k
            tris.append((a, b, c)); tris.append((a, c, d))
    for k in range(n_omega):
        tris.append((bot, k, (k + 1) % n_omega))
        tris.append((top, (nr - 1) * n_omega + k, (nr - 1) * n_omega + (k + 1) % n_omega))
    P, T = np.array(pts, np.float64), np.array(tris, np.int64)
    T = _orient_outward(P, T, (0.0, 0.0, a3))
    # inscribed cylinder: |z - a3| <= 0.8 a3; cross-section radius shrinks
    # with |z|, take it at the first tessellated ring beyond 0.8 a3, and the
    # n_omega-gon chord factor, then shrink by 10%.
    zr = np.abs(z[:, 0] - a3)
    beyond = zr[zr >= 0.8 * a3]
    zb = beyond.min() if beyond.size else a3
    s = min(1.0, zb / a3)
    rho = max(0.0, 1.0 - s ** (2.0 / e1)) ** (e1 / 2.0)
    r = 0.9 * min(a1, a2) * rho * math.cos(math.pi / n_omega)
    # the omega samples are n_omega equal steps: a half turn maps them onto
    # themselves (n_omega even), a quarter turn too when a1 = a2 and 4 | n_omega,
    # and every sample step when the cross-section is a circle (a1 = a2, e2 = 1)
    if a1 == a2 and e2 == 1.0:
        sym = n_omega
    elif a1 == a2 and n_omega % 4 == 0:
        sym = 4
    else:
        sym = 2 if n_omega % 2 == 0 else 1
    return Mesh(name, P.astype(np.float32), T.astype(np.int32), r, 0.2 * a3, 1.8 * a3,
                superquadric_volume(a1, a2, a3, e1, e2), sym)


# ---------------------------------------------------------------------------
# camera, pose grid
# ---------------------------------------------------------------------------
@dataclass
class Camera:
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    T_wc: np.ndarray  # float32 (3, 4): camera -> world, row-major

    @property
    def fxfycxcy(self) -> np.ndarray:
        return np.array([self.fx, self.fy, self.cx, self.cy], np.float32)


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera->world (3x4, float32) for an OpenCV camera (x right, y down,
    z forward) at ``eye`` looking at ``target``."""
    eye, target, up = (np.asarray(v, np.float64) for v in (eye, target, up))
    zc = target - eye; zc /= np.linalg.norm(zc)
    xc = np.cross(zc, up); xc /= np.linalg.norm(xc)
    yc = np.cross(zc, xc)
    T = np.zeros((3, 4))
    T[:, 0], T[:, 1], T[:, 2], T[:, 3] = xc, yc, zc, eye
    return T.astype(np.float32)


@dataclass
class PoseGrid:
    xs: np.ndarray  # float32 (nx,)
    ys: np.ndarray  # float32 (ny,)
    cos_sin: np.ndarray  # float32 (n_yaw, 2)

    @property
    def nx(self): return int(self.xs.shape[0])

    @property
    def ny(self): return int(self.ys.shape[0])

    @property
    def n_yaw(self): return int(self.cos_sin.shape[0])

    @property
    def n_poses(self): return self.nx * self.ny * self.n_yaw


def pose_grid(x0: float, step: float, n: int, n_yaw: int) -> PoseGrid:
    xs = np.array([x0 + step * k for k in range(n)], np.float64).astype(np.float32)
    th = [2.0 * math.pi * k / n_yaw for k in range(n_yaw)]
    cs = np.array([[math.cos(t), math.sin(t)] for t in th], np.float64).astype(np.float32)
    return PoseGrid(xs, xs.copy(), cs)


# object record used by every layer: (mesh, ix, iy, iyaw)
OBJ_DTYPE = np.dtype([("mesh", np.uint16), ("iyaw", np.uint16), ("ix", np.int16), ("iy", np.int16)])


def objs(rows) -> np.ndarray:
    """Object records from (mesh, ix, iy, iyaw) tuples."""
    a = np.zeros(len(rows), OBJ_DTYPE)
    for i, (m, ix, iy, k) in enumerate(rows):
        a[i] = (m, k, ix, iy)
    return a


def all_hypotheses(grid: PoseGrid, meshes_ids) -> np.ndarray:
    """Every (mesh, ix, iy, iyaw) on the grid for the given mesh ids."""
    m = np.asarray(list(meshes_ids), np.int64)
    M, X, Y, K = np.meshgrid(m, np.arange(grid.nx), np.arange(grid.ny), np.arange(grid.n_yaw), indexing="ij")
    a = np.zeros(M.size, OBJ_DTYPE)
    a["mesh"], a["ix"], a["iy"], a["iyaw"] = M.ravel(), X.ravel(), Y.ravel(), K.ravel()
    return a


# ---------------------------------------------------------------------------
# sensor simulation
# ---------------------------------------------------------------------------
_sensor = None


def _load_sensor():
    global _sensor
    if _sensor is None:
        if (not os.path.exists(_SENSOR_LIB)) or os.path.getmtime(_SENSOR_LIB) < os.path.getmtime(_SENSOR_SRC):
            build_sensor()
        lib = ctypes.CDLL(_SENSOR_LIB)
        lib.synth_raycast.restype = ctypes.c_int
        lib.synth_raycast.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p]
        _sensor = lib
    return _sensor


def build_sensor() -> str:
    tmp = _SENSOR_LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SENSOR_SRC, "-lm"])
    os.replace(tmp, _SENSOR_LIB)
    return _SENSOR_LIB


def place(mesh: Mesh, grid: PoseGrid, ix: int, iy: int, iyaw: int) -> np.ndarray:
    """World-frame triangle soup (T, 3, 3) of a placed mesh, in double."""
    v = mesh.verts.astype(np.float64)
    c, s = float(grid.cos_sin[iyaw, 0]), float(grid.cos_sin[iyaw, 1])
    w = np.empty_like(v)
    w[:, 0] = c * v[:, 0] - s * v[:, 1] + float(grid.xs[ix])
    w[:, 1] = s * v[:, 0] + c * v[:, 1] + float(grid.ys[iy])
    w[:, 2] = v[:, 2]
    return w[mesh.tris]


def place_at(mesh: Mesh, x: float, y: float, yaw: float) -> np.ndarray:
    """World-frame triangle soup of a mesh at a continuous pose, in double."""
    v = mesh.verts.astype(np.float64)
    c, s = math.cos(yaw), math.sin(yaw)
    w = np.empty_like(v)
    w[:, 0] = c * v[:, 0] - s * v[:, 1] + x
    w[:, 1] = s * v[:, 0] + c * v[:, 1] + y
    w[:, 2] = v[:, 2]
    return w[mesh.tris]


def _soups(meshes, grid: PoseGrid, scene, jitter=None):
    if jitter is None:
        return [place(meshes[int(o["mesh"])], grid, int(o["ix"]), int(o["iy"]), int(o["iyaw"])) for o in scene]
    out = []
    for o, (dx, dy, dyaw) in zip(scene, np.asarray(jitter, np.float64)):
        yaw = math.atan2(float(grid.cos_sin[o["iyaw"], 1]), float(grid.cos_sin[o["iyaw"], 0])) + dyaw
        out.append(place_at(meshes[int(o["mesh"])], float(grid.xs[o["ix"]]) + dx, float(grid.ys[o["iy"]]) + dy, yaw))
    return out


def raycast_depth(cam: Camera, meshes, grid: PoseGrid, scene, jitter=None) -> np.ndarray:
    """Noise-free sensor depth (float64, H x W, 0 = no return). ``jitter``:
    optional per-object (dx, dy, dyaw) added to the grid poses (objects off
    the grid)."""
    soups = _soups(meshes, grid, scene, jitter)
    tris = np.ascontiguousarray(np.concatenate(soups, 0) if soups else np.zeros((0, 3, 3)), np.float64)
    T = np.ascontiguousarray(cam.T_wc.astype(np.float64))
    out = np.zeros((cam.H, cam.W), np.float64)
    rc = _load_sensor().synth_raycast(cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy,
                                      T.ctypes.data, tris.ctypes.data, tris.shape[0], out.ctypes.data)
    if rc != 0:
        raise RuntimeError("synth_raycast failed")
    return out


def observe(cam: Camera, meshes, grid: PoseGrid, scene, sigma: float, dropout: float, seed: int,
            jitter=None) -> np.ndarray:
    """Simulated observation: ray-cast depth + N(0, sigma^2) on z, then each
    pixel dropped (set to 0 = missing) with probability ``dropout``."""
    d = raycast_depth(cam, meshes, grid, scene, jitter)
    n = d.size
    noise = normal(substream(seed, 1), n).reshape(d.shape)
    drop = uniform(substream(seed, 2), n).reshape(d.shape) < dropout
    valid = d > 0
    d = np.where(valid, d + sigma * noise, 0.0)
    d[drop] = 0.0
    d[d <= 0] = 0.0
    return d.astype(np.float32)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    cam: Camera
    meshes: list
    grid: PoseGrid
    delta: float
    gt: np.ndarray  # OBJ_DTYPE (K,)
    depth: np.ndarray  # float32 (H, W) observation
    sigma: float = 0.0
    dropout: float = 0.0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return int(self.gt.shape[0])

    @property
    def mesh_multiset(self):
        return sorted(int(m) for m in self.gt["mesh"])


def sample_scene(meshes, grid: PoseGrid, mesh_ids, seed: int, margin: float = 0.005,
                 max_tries: int = 100000) -> np.ndarray:
    """Ground-truth objects on the pose grid whose circumscribed footprint
    circles are disjoint (no interpenetration)."""
    k = len(mesh_ids)
    u = uniform(substream(seed, 3), 3 * k * max_tries)
    pos = 0
    for _ in range(max_tries):
        rows = []
        for m in mesh_ids:
            ix = min(int(u[pos] * grid.nx), grid.nx - 1)
            iy = min(int(u[pos + 1] * grid.ny), grid.ny - 1)
            iyaw = min(int(u[pos + 2] * grid.n_yaw), grid.n_yaw - 1)
            pos += 3
            rows.append((m, ix, iy, iyaw))
        ok = True
        for i in range(k):
            for j in range(i + 1, k):
                mi, mj = rows[i], rows[j]
                dx = float(grid.xs[mi[1]]) - float(grid.xs[mj[1]])
                dy = float(grid.ys[mi[2]]) - float(grid.ys[mj[2]])
                rr = meshes[mi[0]].footprint_radius + meshes[mj[0]].footprint_radius + margin
                if dx * dx + dy * dy < rr * rr:
                    ok = False
        if ok:
            return objs(rows)
    raise RuntimeError("could not sample a non-interpenetrating scene")


def camera_c1() -> Camera:
    return Camera(160, 120, 140.0, 140.0, 79.5, 59.5, look_at((0.0, -1.0, 1.0), (0.0, 0.0, 0.0)))


def camera_c2() -> Camera:
    return Camera(640, 480, 525.0, 525.0, 319.5, 239.5, look_at((0.0, -1.0, 1.0), (0.0, 0.0, 0.0)))


def meshes_c1():
    return [box_mesh(0.10, 0.06, 0.15, 9), cylinder_mesh(0.04, 0.12, 64, 15)]


def meshes_c2():
    return [box_mesh(0.10, 0.06, 0.15, 29), cylinder_mesh(0.04, 0.12, 128, 38),
            superquadric_mesh(0.04, 0.04, 0.07, 0.5, 1.0, 51, 100)]


def workload_c1(scene: int = 0, grid: PoseGrid | None = None) -> Workload:
    """160x120, fx=fy=140, box (~1k triangles) + cylinder (~2k), poses on a
    10x10 grid at 5 cm x 8 yaws, sigma = 2 mm, 5% dropout, delta = 1 cm, K = 2."""
    seed = 1000 * 1 + scene
    cam, meshes = camera_c1(), meshes_c1()
    grid = grid or pose_grid(-0.225, 0.05, 10, 8)
    gt = sample_scene(meshes, grid, [0, 1], seed)
    depth = observe(cam, meshes, grid, gt, 0.002, 0.05, seed)
    return Workload("c1", cam, meshes, grid, 0.01, gt, depth, 0.002, 0.05, seed)


def workload_c2(scene: int = 0, grid: PoseGrid | None = None) -> Workload:
    """640x480, fx=fy=525, box / cylinder / superquadric (eps1=0.5, eps2=1)
    of ~10k triangles each, poses on a 50x50 grid at 2 cm x 16 yaws,
    sigma = 3 mm, 5% dropout, delta = 1 cm, K = 3."""
    seed = 1000 * 2 + scene
    cam, meshes = camera_c2(), meshes_c2()
    grid = grid or pose_grid(-0.49, 0.02, 50, 16)
    gt = sample_scene(meshes, grid, [0, 1, 2], seed)
    depth = observe(cam, meshes, grid, gt, 0.003, 0.05, seed)
    return Workload("c2", cam, meshes, grid, 0.01, gt, depth, 0.003, 0.05, seed)


def workload_c2_off_grid(scene: int = 0, off_grid: float = 1.0, grid: PoseGrid | None = None) -> Workload:
    """The C2 camera, meshes and grid with the three objects observed off
    the grid: each at its grid pose plus a uniform offset of up to off_grid/2
    grid steps in x and y and off_grid/2 yaw steps (the recorded ground truth
    stays the grid pose, extra["jitter"] the offsets; footprints 1.5 steps
    further apart), sigma 3 mm, 5% dropout, delta 1 cm."""
    seed = 1000 * 2 + 700 + scene
    cam, meshes = camera_c2(), meshes_c2()
    grid = grid or pose_grid(-0.49, 0.02, 50, 16)
    step = float(grid.xs[1] - grid.xs[0])
    gt = sample_scene(meshes, grid, [0, 1, 2], seed, margin=0.005 + 1.5 * step)
    j = (uniform(substream(seed, 6), 9).reshape(3, 3) - 0.5) * float(off_grid)
    jitter = j * np.array([step, step, 2.0 * math.pi / grid.n_yaw])
    depth = observe(cam, meshes, grid, gt, 0.003, 0.05, seed, jitter)
    return Workload("c2-off-grid", cam, meshes, grid, 0.01, gt, depth, 0.003, 0.05, seed,
                    extra={"jitter": jitter.tolist()})


# ---------------------------------------------------------------------------
# heavy-occlusion workload: eight meshes of uneven size (2k to 50k triangles)
# ---------------------------------------------------------------------------
def prism_mesh(profile, corners, sub: int, n_rings: int, name: str) -> Mesh:
    """Closed solid of revolution-like prism: the boundary polygon `corners`
    (unit circumradius, counter-clockwise), each side split into `sub`
    segments, scaled by profile(z) = (radius, z) at n_rings + 1 heights;
    fan caps. Triangles face outwards."""
    corners = np.asarray(corners, np.float64)
    ring = []
    for k in range(len(corners)):
        a, b = corners[k], corners[(k + 1) % len(corners)]
        for j in range(sub):
            ring.append(a + (b - a) * j / sub)
    ring = np.array(ring)
    n = len(ring)
    pts = []
    for l in range(n_rings + 1):
        r, z = profile(l / n_rings)
        for p in ring:
            pts.append((r * p[0], r * p[1], z))
    top_r, top_z = profile(1.0)
    bot_r, bot_z = profile(0.0)
    top_c = len(pts); pts.append((0.0, 0.0, top_z))
    bot_c = len(pts); pts.append((0.0, 0.0, bot_z))
    tris = []
    for l in range(n_rings):
        for k in range(n):
            a, b = l * n + k, l * n + (k + 1) % n
            c, d = (l + 1) * n + (k + 1) % n, (l + 1) * n + k
            tris.append((a, b, c)); tris.append((a, c, d))
    for k in range(n):
        tris.append((top_c, n_rings * n + k, n_rings * n + (k + 1) % n))
        tris.append((bot_c, (k + 1) % n, k))
    P, T = np.array(pts), np.array(tris, np.int64)
    T = _orient_outward(P, T, (0.0, 0.0, 0.5 * (top_z + bot_z)))
    return P, T


def _ngon(k: int):
    return [(math.cos(2 * math.pi * j / k), math.sin(2 * math.pi * j / k)) for j in range(k)]


def frustum_mesh(r_bot: float, r_top: float, h: float, n_seg: int, n_rings: int, name: str = "frustum") -> Mesh:
    P, T = prism_mesh(lambda t: (r_bot + (r_top - r_bot) * t, h * t), _ngon(n_seg), 1, n_rings, name)
    r = 0.9 * min(r_bot, r_top) * math.cos(math.pi / n_seg)
    return Mesh(name, P.astype(np.float32), T.astype(np.int32), r, 0.05 * h, 0.95 * h, None, n_seg)


def hex_prism_mesh(R: float, h: float, sub: int, n_rings: int, name: str = "hexprism") -> Mesh:
    P, T = prism_mesh(lambda t: (R, h * t), _ngon(6), sub, n_rings, name)
    r = 0.9 * R * math.cos(math.pi / 6)
    return Mesh(name, P.astype(np.float32), T.astype(np.int32), r, 0.05 * h, 0.95 * h, prism_volume(R, 6, h), 6)


def superquadric_general(a1, a2, a3, e1, e2, n_eta, n_omega, name):
    """Superquadric with e2 <= 1 (cross-sections contain the circle of radius
    min(a1, a2) rho(z)); inscribed cylinder shrunk by 15% for tessellation."""
    m = superquadric_mesh(a1, a2, a3, e1, e2, n_eta, n_omega, name)
    z = m.verts[:, 2].astype(np.float64)
    zr = np.abs(z - a3)
    beyond = zr[zr >= 0.8 * a3]
    zb = beyond.min() if beyond.size else a3
    s = min(1.0, zb / a3)
    rho = max(0.0, 1.0 - s ** (2.0 / e1)) ** (e1 / 2.0)
    m.vol_r = 0.85 * min(a1, a2) * rho * math.cos(math.pi / n_omega)
    return m


def meshes_c3():
    """Eight procedural objects of uneven size (2k to 50k triangles) and
    height (6 to 22 cm), so that tall objects can hide short ones."""
    return [
        box_mesh(0.08, 0.06, 0.06, 13, "box2k"),
        cylinder_mesh(0.035, 0.22, 96, 25, "cylinder5k"),
        superquadric_general(0.04, 0.04, 0.045, 0.5, 1.0, 41, 100, "superquadric8k"),
        superquadric_general(0.05, 0.035, 0.03, 1.0, 0.5, 61, 100, "pillow12k"),
        superquadric_general(0.045, 0.04, 0.04, 1.0, 1.0, 91, 100, "ellipsoid18k"),
        frustum_mesh(0.045, 0.03, 0.18, 250, 49, "frustum25k"),
        hex_prism_mesh(0.045, 0.10, 48, 60, "hexprism35k"),
        superquadric_general(0.04, 0.04, 0.035, 0.4, 0.4, 126, 200, "cube50k"),
    ]


def raycast_ids(cam: Camera, meshes, grid: PoseGrid, scene):
    """Noise-free depth (float64) and the index into `scene` of the object
    seen at every pixel (-1 = none)."""
    soups = [place(meshes[int(o["mesh"])], grid, int(o["ix"]), int(o["iy"]), int(o["iyaw"])) for o in scene]
    ids = np.concatenate([np.full(len(s), i, np.int32) for i, s in enumerate(soups)]) if soups else np.zeros(0, np.int32)
    tris = np.ascontiguousarray(np.concatenate(soups, 0) if soups else np.zeros((0, 3, 3)), np.float64)
    T = np.ascontiguousarray(cam.T_wc.astype(np.float64))
    depth = np.zeros((cam.H, cam.W), np.float64)
    obj = np.zeros((cam.H, cam.W), np.int32)
    lib = _load_sensor()
    fn = lib.synth_raycast_ids
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4 + [ctypes.c_void_p] * 2 + [
        ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    ids = np.ascontiguousarray(ids)
    if fn(cam.W, cam.H, cam.fx, cam.fy, cam.cx, cam.cy, T.ctypes.data, tris.ctypes.data, tris.shape[0],
          ids.ctypes.data, depth.ctypes.data, obj.ctypes.data) != 0:
        raise RuntimeError("synth_raycast_ids failed")
    return depth, obj


def occlusion_fractions(cam: Camera, meshes, grid: PoseGrid, scene) -> np.ndarray:
    """Per object: 1 - (pixels where it is the visible surface of the whole
    scene) / (pixels it covers when alone)."""
    _, obj = raycast_ids(cam, meshes, grid, scene)
    out = np.zeros(len(scene))
    for i in range(len(scene)):
        alone = (raycast_ids(cam, meshes, grid, scene[i:i + 1])[1] >= 0).sum()
        out[i] = 1.0 - (obj == i).sum() / max(1, alone)
    return out


def workload_c3(scene: int = 0, grid: PoseGrid | None = None, min_occlusion: float = 0.7) -> Workload:
    """640x480, fx=fy=525; five of the eight uneven meshes, footprints
    disjoint, one of them placed just behind a taller one (as seen from the
    camera) so that at least one object is more than 70% (and less than 100%)
    occluded; poses on the 50x50 x 16-yaw grid; sigma 3 mm, 5% dropout,
    delta 1 cm."""
    seed = 1000 * 3 + scene
    cam, meshes = camera_c2(), meshes_c3()
    grid = grid or pose_grid(-0.49, 0.02, 50, 16)
    step = float(grid.xs[1] - grid.xs[0])
    height = [float(m.verts[:, 2].max()) for m in meshes]
    u = uniform(substream(seed, 4), 200000)
    pos = 0

    def take():
        nonlocal pos
        pos += 1
        return u[pos - 1]

    def disjoint(rows):
        for i in range(len(rows)):
            for j in range(i + 1, len(rows)):
                dx = float(grid.xs[rows[i][1]]) - float(grid.xs[rows[j][1]])
                dy = float(grid.ys[rows[i][2]]) - float(grid.ys[rows[j][2]])
                rr = meshes[rows[i][0]].footprint_radius + meshes[rows[j][0]].footprint_radius + 0.005
                if dx * dx + dy * dy < rr * rr:
                    return False
        return True

    for attempt in range(400):
        ids = np.argsort(u[pos:pos + 8]).tolist()
        pos += 8
        ids = ids[:5]
        front = max(ids, key=lambda m: height[m])  # tallest chosen object in front
        back = [m for m in ids if m != front][int(take() * 4)]
        fx_, fy_ = 15 + int(take() * 20), 12 + int(take() * 12)
        gap = meshes[front].footprint_radius + meshes[back].footprint_radius + 0.006
        by = fy_ + int(math.ceil(gap / step)) + int(take() * 2)
        bx = fx_ + int(take() * 3) - 1
        rows = [(front, fx_, fy_, int(take() * grid.n_yaw)), (back, bx, by, int(take() * grid.n_yaw))]
        for m in ids:
            if m in (front, back):
                continue
            for _ in range(50):
                cand = (m, 10 + int(take() * 30), 8 + int(take() * 34), int(take() * grid.n_yaw))
                if disjoint(rows + [cand]):
                    rows.append(cand)
                    break
        if len(rows) < 5 or not disjoint(rows) or max(by, bx) >= grid.ny:
            continue
        gt = objs(sorted(rows))
        occ = occlusion_fractions(cam, meshes, grid, gt)
        if occ.max() > min_occlusion and occ.max() < 1.0:
            depth = observe(cam, meshes, grid, gt, 0.003, 0.05, seed)
            return Workload("c3", cam, meshes, grid, 0.01, gt, depth, 0.003, 0.05, seed,
                            extra={"occlusion": occ.tolist()})
    raise RuntimeError("no heavily occluded scene found")


def workload_c3_reduced(scene: int = 0, grid: PoseGrid | None = None, k: int = 3,
                        min_occlusion: float = 0.3) -> Workload:
    """The heavy-occlusion setting on a coarse pose grid, small enough for
    the oracle's exact search: 640x480, k of the eight uneven meshes, the
    tallest chosen one placed at a random cell and another one in the nearest
    row behind it (as seen from the camera) whose footprint stays disjoint,
    the rest anywhere disjoint; a scene is kept when some object is more than
    min_occlusion (and less than 100%) occluded. Default grid 8 x 8 positions
    (0.14 m apart) x 4 yaws; sigma 3 mm, 5% dropout, delta 1 cm."""
    seed = 1000 * 3 + 500 + scene
    cam, meshes = camera_c2(), meshes_c3()
    grid = grid or pose_grid(-0.49, 0.14, 8, 4)
    height = [float(m.verts[:, 2].max()) for m in meshes]
    u = uniform(substream(seed, 7), 100000)
    pos = 0

    def take():
        nonlocal pos
        pos += 1
        return u[pos - 1]

    def disjoint(rows):
        for i in range(len(rows)):
            for j in range(i + 1, len(rows)):
                dx = float(grid.xs[rows[i][1]]) - float(grid.xs[rows[j][1]])
                dy = float(grid.ys[rows[i][2]]) - float(grid.ys[rows[j][2]])
                rr = meshes[rows[i][0]].footprint_radius + meshes[rows[j][0]].footprint_radius + 0.005
                if dx * dx + dy * dy < rr * rr:
                    return False
        return True

    for _ in range(400):
        ids = np.argsort(u[pos:pos + len(meshes)]).tolist()[:k]
        pos += len(meshes)
        front = max(ids, key=lambda m: height[m])
        back = [m for m in ids if m != front][min(int(take() * (k - 1)), k - 2)]
        fx_, fy_ = min(int(take() * grid.nx), grid.nx - 1), min(int(take() * (grid.ny - 1)), grid.ny - 2)
        rows = [(front, fx_, fy_, min(int(take() * grid.n_yaw), grid.n_yaw - 1))]
        for by in range(fy_ + 1, grid.ny):
            cand = (back, fx_, by, min(int(take() * grid.n_yaw), grid.n_yaw - 1))
            if disjoint(rows + [cand]):
                rows.append(cand)
                break
        for m in ids:
            if m in (front, back):
                continue
            for _ in range(50):
                cand = (m, min(int(take() * grid.nx), grid.nx - 1), min(int(take() * grid.ny), grid.ny - 1),
                        min(int(take() * grid.n_yaw), grid.n_yaw - 1))
                if disjoint(rows + [cand]):
                    rows.append(cand)
                    break
        if len(rows) < k:
            continue
        gt = objs(sorted(rows))
        occ = occlusion_fractions(cam, meshes, grid, gt)
        if min_occlusion < occ.max() < 1.0:
            depth = observe(cam, meshes, grid, gt, 0.003, 0.05, seed)
            return Workload("c3-reduced", cam, meshes, grid, 0.01, gt, depth, 0.003, 0.05, seed,
                            extra={"occlusion": occ.tolist()})
    raise RuntimeError("no occluded scene found")


def workloads_c5(n_scenes: int = 256, grid: PoseGrid | None = None, cam: Camera | None = None, meshes=None,
                 k_range=(2, 6), seed_base: int = 5000, first: int = 0, off_grid: float = 0.0):
    """Many independent scenes for concurrent search: scene s draws K uniform
    in k_range and K distinct meshes of the eight uneven ones, poses anywhere
    on the grid with disjoint footprints; 640x480 by default, sigma 3 mm,
    5% dropout, delta 1 cm. Scene s is seeded with seed_base + s (s from
    ``first``); disjoint seed ranges give disjoint scene sets (training scenes
    of the learned heuristic: 7000 + s; its held-out 5-object scenes: 9000 + s).
    off_grid = a in (0, 1]: the observed objects sit at their grid pose plus
    a uniform offset of up to a/2 grid steps in x and y and a/2 yaw steps (the
    recorded ground truth stays the grid pose, extra["jitter"] the offsets);
    footprints are then kept 1.5 grid steps further apart."""
    cam = cam or camera_c2()
    meshes = meshes or meshes_c3()
    grid = grid or pose_grid(-0.49, 0.02, 50, 16)
    out = []
    for s in range(first, first + n_scenes):
        seed = seed_base + s
        u = uniform(substream(seed, 5), 16)
        K = k_range[0] + min(int(u[0] * (k_range[1] - k_range[0] + 1)), k_range[1] - k_range[0])
        ids = sorted(np.argsort(u[1:1 + len(meshes)])[:K].tolist())
        step = float(grid.xs[1] - grid.xs[0]) if grid.nx > 1 else 0.0
        jitter = None
        if off_grid:
            gt = sample_scene(meshes, grid, ids, seed, margin=0.005 + 1.5 * step)
            j = (uniform(substream(seed, 6), 3 * K).reshape(K, 3) - 0.5) * float(off_grid)
            jitter = j * np.array([step, step, 2.0 * math.pi / grid.n_yaw])
        else:
            gt = sample_scene(meshes, grid, ids, seed)
        depth = observe(cam, meshes, grid, gt, 0.003, 0.05, seed, jitter)
        extra = {} if jitter is None else {"jitter": jitter.tolist()}
        out.append(Workload(f"c5/{s}", cam, meshes, grid, 0.01, gt, depth, 0.003, 0.05, seed, extra=extra))
    return out


# ---------------------------------------------------------------------------
# seeded initial weights of the learned heuristic's network
# ---------------------------------------------------------------------------
def he_normal(shapes, seed: int):
    """One float32 array per shape: arrays of rank > 1 are weights, drawn
    normal with variance 2 / fan_in (fan_in = product of all but the first
    dimension); rank-1 arrays (biases) are zero. Array i uses sub-stream i."""
    out = []
    for i, shp in enumerate(shapes):
        n = int(np.prod(shp))
        if len(shp) > 1:
            fan_in = int(np.prod(shp[1:]))
            a = normal(substream(seed, 100 + i), n) * math.sqrt(2.0 / fan_in)
        else:
            a = np.zeros(n)
        out.append(a.reshape(shp).astype(np.float32))
    return out
