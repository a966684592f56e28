"""Pose accuracy of a returned scene against the ground truth.

Sec. V-D's criterion: a predicted pose (x, y, theta) of an object is correct
when ||(x, y) - (x_true, y_true)|| < dt and the shortest angular difference
between theta and theta_true is < dtheta. For an object whose mesh is
invariant under a turn of 2 pi / sym about its vertical axis, yaws that
differ by a multiple of 2 pi / sym are the same pose (Sec. IV-E: only (x, y)
matters for a rotationally symmetric object), so the angular difference is
taken modulo 2 pi / sym. Predicted and true objects of the same type are
paired by the assignment of smallest total position error.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

DT_M = (0.01, 0.02, 0.05, 0.1)
DTHETA_DEG = (5.0, 10.0, 22.5, 180.0)


def yaw_angle(grid, iyaw: int) -> float:
    """The yaw of a grid index, from the pose table's (cos, sin) in double."""
    c, s = (float(v) for v in grid.cos_sin[int(iyaw)])
    return math.atan2(s, c)


def angular_difference(a: float, b: float, sym: int = 1) -> float:
    """Shortest angular difference (radians) between yaws a and b, modulo
    2 pi / sym."""
    period = 2.0 * math.pi / max(int(sym), 1)
    d = math.fmod(abs(a - b), period)
    return min(d, period - d)


def true_poses(wl):
    """(mesh, x, y, yaw) of the workload's observed objects: the ground-truth
    grid poses plus the off-grid offsets the observation was made with."""
    jit = wl.extra.get("jitter") if wl.extra else None
    out = []
    for k, o in enumerate(wl.gt):
        x, y = float(wl.grid.xs[o["ix"]]), float(wl.grid.ys[o["iy"]])
        yaw = yaw_angle(wl.grid, o["iyaw"])
        if jit is not None:
            x, y, yaw = x + jit[k][0], y + jit[k][1], yaw + jit[k][2]
        out.append((int(o["mesh"]), x, y, yaw))
    return out


def pose_errors(pred, truth, grid, syms):
    """Per true object: (mesh, position error in m, yaw error in degrees),
    pairing predicted objects (OBJ records on `grid`) with true poses of the
    same mesh by the permutation of smallest total position error; a true
    object without a prediction of its type gets (mesh, inf, inf)."""
    poses = [(int(o["mesh"]), float(grid.xs[o["ix"]]), float(grid.ys[o["iy"]]), yaw_angle(grid, o["iyaw"]))
             for o in pred]
    return pose_errors_of(poses, truth, syms)


def pose_errors_of(poses, truth, syms):
    """pose_errors for predicted poses given as (mesh, x, y, yaw) (off the
    grid, e.g. refined by ICP)."""
    out = []
    for m in sorted({t[0] for t in truth}):
        T = [t for t in truth if t[0] == m]
        P = [(x, y, yaw) for mm, x, y, yaw in poses if int(mm) == m]
        best, best_cost = None, math.inf
        n = min(len(T), len(P))
        for perm in itertools.permutations(range(len(P)), n):
            cost = sum(math.hypot(P[j][0] - T[i][1], P[j][1] - T[i][2]) for i, j in enumerate(perm))
            if cost < best_cost:
                best, best_cost = perm, cost
        for i, t in enumerate(T):
            if best is None or i >= n:
                out.append((m, math.inf, math.inf))
                continue
            p = P[best[i]]
            dt = math.hypot(p[0] - t[1], p[1] - t[2])
            dth = math.degrees(angular_difference(p[2], t[3], syms[m]))
            out.append((m, dt, dth))
    return out


def correct_counts(errors, dts=DT_M, dthetas=DTHETA_DEG):
    """{(dt, dtheta): number of objects within both thresholds} (strict <)."""
    return {(dt, dth): sum(1 for _, e, a in errors if e < dt and a < dth) for dt in dts for dth in dthetas}


def report(results, workloads, meshes):
    """Accuracy of the scenes a search returned (one result dict per
    workload, as perch_search / perch_search_multi give them): the number of
    objects, the counts within every (dt, dtheta) pair, and the mean errors of
    the objects found within 10 cm."""
    syms = [int(getattr(m, "sym", 1)) for m in meshes]
    errs = []
    for r, wl in zip(results, workloads):
        errs += pose_errors(r["objs"], true_poses(wl), wl.grid, syms)
    counts = correct_counts(errs)
    near = [(e, a) for _, e, a in errs if e < 0.1]
    return {"objects": len(errs),
            "correct": {f"{dt * 100:g}cm/{dth:g}deg": c for (dt, dth), c in counts.items()},
            "mean_position_error_m": float(np.mean([e for e, _ in near])) if near else None,
            "mean_yaw_error_deg": float(np.mean([a for _, a in near])) if near else None,
            "criterion": "Sec. V-D: position error < dt and shortest yaw difference (modulo the mesh's "
                         "rotational symmetry) < dtheta"}
