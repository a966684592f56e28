"""Pins of the oracle's closed-form object volumes V(O) (Sec. III-A: the set
of points in the volume the object occupies, in closed form where there is
one; the inscribed cylinder is the conservative stand-in otherwise).

The reference is the mesh itself: every mesh with a closed form here is
convex, so the volume it occupies is the convex hull of its vertices, taken
in float64 by Qhull (scipy.spatial.ConvexHull), an implementation that shares
nothing with the oracle. Points are placed around each object at several
yaws of the pose grid (so a wrong rotation sign or a swapped axis moves the
box's long side) and carried into the world frame in float64:
  - box and regular prism: the closed form is the mesh's solid, so a point
    farther than 1e-6 m inside the hull is in V(O) and one farther than
    1e-6 m outside is not;
  - superquadric / ellipsoid: the mesh is a tessellation with its vertices on
    the surface, so the closed-form solid holds the hull; a point inside the
    hull is in V(O), and one more than 2 mm outside it is not.
Then the decomposition identities that hold for any V(O) are checked with
the closed forms on: the K = 1 identity with the undecomposed cost and the
zero-cost ground-truth path on a noise-free observation.
"""
import numpy as np
import pytest

import oracle
from paper_1510_05613_gb300 import synth

spatial = pytest.importorskip("scipy.spatial")

MESHES = [m for m in synth.meshes_c2() + synth.meshes_c3() if m.volume is not None]


def _hull(m):
    h = spatial.ConvexHull(m.verts.astype(np.float64))
    return h.equations  # rows (n, d): n . p + d <= 0 inside


def _points(m, rng, n=4000):
    v = m.verts.astype(np.float64)
    lo, hi = v.min(0), v.max(0)
    pad = 0.15 * (hi - lo)
    pts = rng.uniform(lo - pad, hi + pad, (n, 3))
    # and points right at the surface, pushed in and out along the radius
    on = v[rng.choice(len(v), n // 4)]
    c = np.array([0.0, 0.0, 0.5 * (lo[2] + hi[2])])
    for f in (0.995, 1.005):
        pts = np.concatenate([pts, c + (on - c) * f])
    return pts


@pytest.mark.parametrize("m", MESHES, ids=[m.name for m in MESHES])
def test_closed_form_volume_matches_the_mesh_hull(m):
    rng = np.random.default_rng(17)
    grid = synth.pose_grid(-0.2, 0.1, 5, 16)
    meshes = [m]
    cam = synth.camera_c2()
    w = oracle.World(cam, meshes, grid, 0.01, exact_volumes=True)
    eq = _hull(m)
    P = _points(m, rng)
    dist = (P @ eq[:, :3].T + eq[:, 3]).max(1)  # > 0 outside the hull, < 0 inside (distance to the nearest face plane)
    sq = m.volume.kind == synth.VOL_SUPERQUADRIC
    n_in = n_out = 0
    for iyaw in (0, 1, 3, 5, 6):
        ix, iy = 1, 3
        cs, sn = (float(v) for v in grid.cos_sin[iyaw])
        # object frame -> world, float64: rotate by yaw, translate by the grid position
        world = np.stack([cs * P[:, 0] - sn * P[:, 1] + float(grid.xs[ix]),
                          sn * P[:, 0] + cs * P[:, 1] + float(grid.ys[iy]), P[:, 2]], 1)
        got = oracle.in_volume(w, synth.objs([(0, ix, iy, iyaw)])[0], world)
        inside = dist < -1e-6
        outside = dist > (2e-3 if sq else 1e-6)
        assert got[inside].all(), (m.name, iyaw, P[inside & (got == 0)][:3])
        assert not got[outside].any(), (m.name, iyaw, P[outside & (got == 1)][:3])
        n_in += inside.sum()
        n_out += outside.sum()
    assert n_in > 1000 and n_out > 1000


def test_closed_form_volume_is_larger_than_the_inscribed_cylinder():
    """The inscribed cylinder is a subset of the closed form (it is the
    conservative stand-in of Sec. III-A), and the closed form holds strictly
    more of the object's own surface points pushed 1 mm inwards."""
    for m in MESHES:
        grid = synth.pose_grid(0.0, 0.1, 1, 8)
        cam = synth.camera_c2()
        we = oracle.World(cam, [m], grid, 0.01, exact_volumes=True)
        wc = oracle.World(cam, [m], grid, 0.01, exact_volumes=False)
        v = m.verts.astype(np.float64)
        c = np.array([0.0, 0.0, 0.5 * v[:, 2].max()])
        d = v - c
        inner = v - 1e-3 * d / np.linalg.norm(d, axis=1, keepdims=True)
        o = synth.objs([(0, 0, 0, 3)])[0]
        cs, sn = (float(x) for x in grid.cos_sin[3])
        world = np.stack([cs * inner[:, 0] - sn * inner[:, 1], sn * inner[:, 0] + cs * inner[:, 1], inner[:, 2]], 1)
        e, cyl = oracle.in_volume(we, o, world), oracle.in_volume(wc, o, world)
        assert (e >= cyl).all(), m.name
        assert e.sum() > cyl.sum() + 0.3 * len(v), (m.name, e.sum(), cyl.sum(), len(v))


@pytest.fixture(scope="module")
def c1():
    return synth.workload_c1()


def test_k1_decomposition_with_closed_form_volumes(c1):
    """K = 1: dJr = J_r and dJo + residual = J_o for any V(O) (Sec. IV-A)."""
    w = oracle.World.of(c1, exact_volumes=True)
    rng = np.random.default_rng(6)
    hyps = synth.all_hypotheses(c1.grid, [0, 1])
    pick = np.concatenate([hyps[rng.choice(len(hyps), 40, replace=False)], c1.gt])
    recs = oracle.eval_batch(w, c1.depth, [pick[:0]], np.zeros(len(pick), np.int32), pick, 1)
    wc = oracle.World.of(c1)
    recs_c = oracle.eval_batch(wc, c1.depth, [pick[:0]], np.zeros(len(pick), np.int32), pick, 1)
    for h, r in zip(pick, recs):
        jo, jr = oracle.cost_J(w, c1.depth, np.array([h]))
        assert r[0] == jr and r[1] + r[2] == jo
    # the closed form holds the inscribed cylinder: at least as many observed
    # points in V(O) for every hypothesis, more for many
    assert (recs[:, 6] >= recs_c[:, 6]).all() and (recs[:, 6] > recs_c[:, 6]).sum() > 5


@pytest.mark.parametrize("wl_fn", [synth.workload_c1, synth.workload_c2])
def test_ground_truth_path_zero_cost_with_closed_form_volumes(wl_fn):
    wl = wl_fn()
    w = oracle.World.of(wl, exact_volumes=True)
    z, _ = oracle.render(w, wl.gt)
    depth = np.where(np.isfinite(z), z, 0).astype(np.float32)
    order = wl.gt
    total = 0
    for j in range(len(order)):
        r = oracle.eval_batch(w, depth, [order[:j]], np.zeros(1, np.int32), order[j:j + 1], wl.K)[0]
        if r[3] > 0:
            pytest.skip("this order is not front to back")
        total += int(r[0] + r[1] + r[2])
    assert total == 0
