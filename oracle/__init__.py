"""PERCH CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never loads it and shares no code with it.

``perch_oracle.c`` is a plain restatement of the paper's definitions
(Eq. (1) explanation indicator, Sec. III-B explanation cost, Sec. IV-A
decomposition into per-edge costs, Eq. (3)/(4) monotone successors and edge
cost); ``search.py`` holds the plain tree searches (uniform-cost search over
the MSGT of Sec. IV-A/B, and exhaustive enumeration for tiny inputs).

Pins (tests/test_oracle_*.py): the observed cloud's camera and world points
against float64 pinhole back-projection and sensor pose (a camera with
fx != fy, cx != cy, a non-square image; the table plane and ray-cast box faces),
closed-form depths of single triangles and box faces, the watertightness invariant of the coverage rule, brute-force
point-in-triangle coverage with exact rationals, exact-delta ties of Eq. (1),
the K = 1 identity between the decomposed and undecomposed cost, the
zero-cost ground-truth path on a noise-free observation, empty-observation and
infinite-delta special cases, and search == exhaustive enumeration.
The ICP refinement of Sec. IV-E-1 (tests/test_oracle_icp.py): the planar
fit against known motions and an SVD fit, the correspondence rule against
brute-force and k-d tree nearest neighbours, the model set against the edge
cost's |dR|, the exact identity on an observation that is the object's own
render, and off-grid objects of the ray-cast sensor brought to their true
pose.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "perch_oracle.c")
_LIB = os.path.join(_HERE, "libperch_oracle.so")

REC_FIELDS = ("djr", "djo", "resid", "viol", "n_new", "flags", "n_vol")
FLAG_CULLED, FLAG_INVALID = 1, 2
# ICP record (Sec. IV-E-1): the planar motion (c, s, tx, ty), |M|, the last
# matching's pairs, the fits made, and how the iteration stopped
ICP_DTYPE = np.dtype([("c", "<f8"), ("s", "<f8"), ("tx", "<f8"), ("ty", "<f8"), ("n_model", "<i4"),
                      ("n_corr", "<i4"), ("iters", "<i4"), ("status", "<i4")])
ICP_CONVERGED, ICP_CAP, ICP_FEW, ICP_DEGENERATE = 0, 1, 2, 3


def build() -> str:
    """Compile the oracle (IEEE binary32 ops, no FMA contraction)."""
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Mesh(ctypes.Structure):
    _fields_ = [("n_verts", ctypes.c_int32), ("n_tris", ctypes.c_int32),
                ("verts", ctypes.c_void_p), ("tris", ctypes.c_void_p),
                ("vol_r", ctypes.c_float), ("vol_zlo", ctypes.c_float), ("vol_zhi", ctypes.c_float),
                ("kind", ctypes.c_int32), ("n", ctypes.c_int32), ("p", ctypes.c_float * 4),
                ("zlo", ctypes.c_float), ("zhi", ctypes.c_float), ("normals", ctypes.c_void_p)]


class _World(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("T_wc", ctypes.c_float * 12),
                ("xs", ctypes.c_void_p), ("nx", ctypes.c_int32),
                ("ys", ctypes.c_void_p), ("ny", ctypes.c_int32),
                ("cos_sin", ctypes.c_void_p), ("n_yaw", ctypes.c_int32),
                ("meshes", ctypes.c_void_p), ("n_mesh", ctypes.c_int32),
                ("delta", ctypes.c_float)]


class _ObjArg(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_uint16), ("iyaw", ctypes.c_uint16), ("ix", ctypes.c_int16), ("iy", ctypes.c_int16)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            build()
        lib = ctypes.CDLL(_LIB)
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.or_render.restype = I64
        lib.or_render.argtypes = [P, P, I32, P]
        lib.or_observed.restype = I64
        lib.or_observed.argtypes = [P, P, P, P]
        lib.or_unexplained.restype = I32
        lib.or_unexplained.argtypes = [P, I64, P, I64, ctypes.c_float, P]
        lib.or_cost_J.restype = I32
        lib.or_cost_J.argtypes = [P, P, P, I32, P]
        lib.or_eval_batch.restype = I32
        lib.or_eval_batch.argtypes = [P, P, P, P, I32, I32, P, P, I64, I32, P, I32]
        lib.or_max_threads.restype = I32
        lib.or_in_volume.restype = I32
        lib.or_in_volume.argtypes = [P, _ObjArg, P, I64, P]
        lib.or_icp_refine.restype = I32
        lib.or_icp_refine.argtypes = [P, P, P, P, I32, I32, P, P, I64, ctypes.c_float, I32, P, I32]
        lib.or_icp_fit.restype = I32
        lib.or_icp_fit.argtypes = [P, P, I64, P]
        lib.or_icp_match.restype = I32
        lib.or_icp_match.argtypes = [P, P, P, I64, ctypes.c_float, P]
        _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class World:
    """Camera, meshes, pose tables and delta, as the oracle sees them."""

    def __init__(self, cam, meshes, grid, delta: float, exact_volumes: bool = False):
        """``exact_volumes``: V(O) is each mesh's closed-form solid where it
        has one (mesh.volume), else the inscribed cylinder."""
        self._keep = []
        ms = (_Mesh * max(1, len(meshes)))()
        for i, m in enumerate(meshes):
            v, t = _c(m.verts, np.float32), _c(m.tris, np.int32)
            self._keep += [v, t]
            ms[i] = _Mesh(m.n_verts, m.n_tris, v.ctypes.data, t.ctypes.data, m.vol_r, m.vol_zlo, m.vol_zhi)
            vol = getattr(m, "volume", None)
            if exact_volumes and vol is not None:
                nr = _c(vol.normals, np.float32)
                self._keep.append(nr)
                ms[i].kind, ms[i].n = int(vol.kind), int(vol.n)
                for k in range(4):
                    ms[i].p[k] = float(np.float32(vol.p[k]))
                ms[i].zlo, ms[i].zhi = float(vol.zlo), float(vol.zhi)
                ms[i].normals = nr.ctypes.data if nr.size else None
        self._keep.append(ms)
        xs, ys, cs = _c(grid.xs, np.float32), _c(grid.ys, np.float32), _c(grid.cos_sin, np.float32)
        self._keep += [xs, ys, cs]
        w = _World()
        w.W, w.H = cam.W, cam.H
        w.fx, w.fy, w.cx, w.cy = cam.fx, cam.fy, cam.cx, cam.cy
        for k, val in enumerate(np.asarray(cam.T_wc, np.float32).reshape(-1)):
            w.T_wc[k] = float(val)
        w.xs, w.nx = xs.ctypes.data, xs.shape[0]
        w.ys, w.ny = ys.ctypes.data, ys.shape[0]
        w.cos_sin, w.n_yaw = cs.ctypes.data, cs.shape[0]
        w.meshes, w.n_mesh = ctypes.addressof(ms), len(meshes)
        w.delta = delta
        self.c = w
        self.W, self.H = cam.W, cam.H
        self.delta = delta
        self.n_mesh = len(meshes)

    @classmethod
    def of(cls, wl, delta=None, exact_volumes: bool = False):
        return cls(wl.cam, wl.meshes, wl.grid, wl.delta if delta is None else delta, exact_volumes)

    def ptr(self):
        return ctypes.addressof(self.c)


def _objs(a):
    from paper_1510_05613_gb300.synth import OBJ_DTYPE
    return np.ascontiguousarray(np.asarray(a, OBJ_DTYPE))


def render(world: World, objs):
    """(z-buffer float32 H x W with +inf where empty, culled-triangle count)."""
    o = _objs(objs)
    z = np.empty((world.H, world.W), np.float32)
    culled = _load().or_render(world.ptr(), o.ctypes.data, len(o), z.ctypes.data)
    if culled < 0:
        raise MemoryError("oracle render")
    return z, int(culled)


def observed(world: World, depth):
    """Observed cloud I: (camera-frame (n,3), world-frame (n,3)) float32."""
    d = _c(depth, np.float32)
    cam = np.empty((world.W * world.H, 3), np.float32)
    wor = np.empty_like(cam)
    n = _load().or_observed(world.ptr(), d.ctypes.data, cam.ctypes.data, wor.ctypes.data)
    return cam[:n].copy(), wor[:n].copy()


def unexplained(P, Q, delta: float):
    """Eq. (1) indicator for each row of P against cloud Q (both (n,3))."""
    P, Q = _c(P, np.float32).reshape(-1, 3), _c(Q, np.float32).reshape(-1, 3)
    out = np.empty(P.shape[0], np.int32)
    _load().or_unexplained(P.ctypes.data, P.shape[0], Q.ctypes.data, Q.shape[0], delta, out.ctypes.data)
    return out


def cost_J(world: World, depth, objs):
    """Undecomposed (J_o, J_r) of a full assignment (Sec. III-B)."""
    o = _objs(objs)
    d = _c(depth, np.float32)
    out = np.zeros(2, np.int64)
    if _load().or_cost_J(world.ptr(), d.ctypes.data, o.ctypes.data, len(o), out.ctypes.data):
        raise MemoryError("oracle cost_J")
    return int(out[0]), int(out[1])


def eval_batch(world: World, depth, parents, hyp_parent, hyps, K_total: int, threads: int = 0):
    """Edge-cost records (n_hyp, 7) int32: dJr, dJo, resid, viol, n_new, flags,
    n_vol (observed points newly inside the assigned volumes).

    ``parents`` is a list of object arrays (each a partial assignment)."""
    from paper_1510_05613_gb300.synth import OBJ_DTYPE
    k_max = max([1] + [len(p) for p in parents])
    P = np.zeros((max(1, len(parents)), k_max), OBJ_DTYPE)
    plen = np.zeros(max(1, len(parents)), np.int32)
    for i, p in enumerate(parents):
        P[i, :len(p)] = p
        plen[i] = len(p)
    hp = _c(hyp_parent, np.int32)
    h = _objs(hyps)
    d = _c(depth, np.float32)
    recs = np.zeros((len(h), 7), np.int32)
    rc = _load().or_eval_batch(world.ptr(), d.ctypes.data, P.ctypes.data, plen.ctypes.data, len(parents), k_max,
                               hp.ctypes.data, h.ctypes.data, len(h), K_total, recs.ctypes.data, threads)
    if rc:
        raise MemoryError("oracle eval_batch")
    return recs


def in_volume(world: World, obj, pts):
    """V(O) membership (0/1 per row) of world points (n, 3) for one object."""
    o = _objs([obj])[0]
    q = _c(pts, np.float32).reshape(-1, 3)
    out = np.empty(q.shape[0], np.int32)
    _load().or_in_volume(world.ptr(), _ObjArg(int(o["mesh"]), int(o["iyaw"]), int(o["ix"]), int(o["iy"])),
                         q.ctypes.data, q.shape[0], out.ctypes.data)
    return out


def max_threads() -> int:
    return int(_load().or_max_threads())


def _parent_table(parents):
    from paper_1510_05613_gb300.synth import OBJ_DTYPE
    k_max = max([1] + [len(p) for p in parents])
    P = np.zeros((max(1, len(parents)), k_max), OBJ_DTYPE)
    plen = np.zeros(max(1, len(parents)), np.int32)
    for i, p in enumerate(parents):
        P[i, :len(p)] = p
        plen[i] = len(p)
    return P, plen, k_max


def icp_refine(world: World, depth, parents, hyp_parent, hyps, radius: float = 0.02, max_iter: int = 20,
               threads: int = 0):
    """ICP refinement of each successor's new object (Sec. IV-E-1): one
    ICP_DTYPE record per hypothesis. ``parents`` as in eval_batch."""
    P, plen, k_max = _parent_table(parents)
    hp = _c(hyp_parent, np.int32)
    h = _objs(hyps)
    d = _c(depth, np.float32)
    out = np.zeros(len(h), ICP_DTYPE)
    rc = _load().or_icp_refine(world.ptr(), d.ctypes.data, P.ctypes.data, plen.ctypes.data, len(parents), k_max,
                               hp.ctypes.data, h.ctypes.data, len(h), float(radius), int(max_iter),
                               out.ctypes.data, threads)
    if rc:
        raise MemoryError("oracle icp_refine")
    return out


def icp_fit(m, q):
    """The closed-form planar fit on explicit pairs (world points (n, 3)):
    ((c, s, tx, ty), status) with status 0 = fitted, 1 = no turn defined,
    2 = fewer than 3 pairs."""
    m, q = _c(m, np.float32).reshape(-1, 3), _c(q, np.float32).reshape(-1, 3)
    out = np.zeros(4, np.float64)
    st = _load().or_icp_fit(m.ctypes.data, q.ctypes.data, m.shape[0], out.ctypes.data)
    return tuple(float(v) for v in out), int(st)


def icp_match(world: World, depth, pts, radius: float):
    """Index in I (pixel order) of each world point's correspondence, -1 if
    none is within ``radius``."""
    p = _c(pts, np.float32).reshape(-1, 3)
    d = _c(depth, np.float32)
    idx = np.empty(p.shape[0], np.int64)
    if _load().or_icp_match(world.ptr(), d.ctypes.data, p.ctypes.data, p.shape[0], float(radius), idx.ctypes.data):
        raise MemoryError("oracle icp_match")
    return idx


def icp_pose(grid, obj, rec):
    """Refined (x, y, yaw) of a grid object moved by an ICP record's motion:
    (x, y) turned and shifted, the yaw turned by atan2(s, c) (double)."""
    import math
    x, y = float(grid.xs[int(obj["ix"])]), float(grid.ys[int(obj["iy"])])
    c0, s0 = (float(v) for v in grid.cos_sin[int(obj["iyaw"])])
    c, s = float(rec["c"]), float(rec["s"])
    return (c * x - s * y + float(rec["tx"]), s * x + c * y + float(rec["ty"]),
            math.atan2(s0, c0) + math.atan2(s, c))
