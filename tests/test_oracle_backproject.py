"""Pins of the oracle's observed cloud I (Sec. III-A): back-projection of the
depth image through the pinhole model into camera points, and the sensor pose
that carries them into the world frame, where V(O) membership and the
overlap heuristic of Sec. IV-C are decided.

Every expected value here is computed in float64 inside the test from
(u, v, d), the intrinsics and T_world_cam -- never from the oracle's own
points -- so a slip in the oracle (ray slope taken with the wrong focal
length, the two slopes swapped, the translation's sign flipped, the rotation
transposed) fails one of them. The camera has fx != fy, cx != cy, a
non-square image and a rotation that is not symmetric, so none of those
slips cancels out.

The binary32 bounds follow from the oracle's operation order: a camera
coordinate is (float)((u - cx) / fx) * d, two roundings, so it is within
(2^-23 + 2^-48) |exact| of the float64 value; a world coordinate adds a
product, two fused multiply-adds and the translation (four more roundings of
quantities bounded by S = sum_k |R_rk| |p_k| + |t_r|).
"""
import numpy as np
import pytest

import oracle
from paper_1510_05613_gb300 import synth

U = 2.0 ** -24  # unit roundoff of binary32


def _camera():
    # off-axis eye, a look-at target away from the origin: every entry of R
    # differs from its transpose partner
    T = synth.look_at((0.31, -0.83, 0.97), (0.05, 0.02, 0.0))
    return synth.Camera(37, 23, 61.25, 47.5, 17.75, 9.5, T)


def _world(cam):
    c1 = synth.workload_c1()
    return oracle.World(cam, c1.meshes, c1.grid, 0.01), c1


def _depth(cam, seed=3):
    rng = np.random.default_rng(seed)
    d = rng.uniform(0.3, 3.0, (cam.H, cam.W)).astype(np.float32)
    holes = rng.random((cam.H, cam.W))
    d[holes < 0.05] = 0.0
    d[(holes >= 0.05) & (holes < 0.07)] = np.nan
    d[(holes >= 0.07) & (holes < 0.08)] = np.inf
    d[(holes >= 0.08) & (holes < 0.09)] = -0.5
    return d


def _exact_camera_points(cam, depth):
    """float64 pinhole back-projection of every valid pixel, row-major."""
    v, u = np.nonzero(np.isfinite(depth) & (depth > 0))
    d = depth[v, u].astype(np.float64)
    x = (u.astype(np.float64) - float(cam.cx)) / float(cam.fx) * d
    y = (v.astype(np.float64) - float(cam.cy)) / float(cam.fy) * d
    return np.stack([x, y, d], 1), u, v


def _exact_world(cam, p):
    T = cam.T_wc.astype(np.float64)
    R, t = T[:, :3], T[:, 3]
    S = np.abs(p) @ np.abs(R).T + np.abs(t)[None, :]
    return p @ R.T + t[None, :], S


def test_camera_points_match_float64_pinhole():
    cam = _camera()
    w, _ = _world(cam)
    depth = _depth(cam)
    got, _ = oracle.observed(w, depth)
    exact, u, v = _exact_camera_points(cam, depth)
    assert got.shape == exact.shape and len(exact) > 600  # every valid pixel, nothing else
    err = np.abs(got.astype(np.float64) - exact)
    bound = (2 * U + U * U) * np.abs(exact)
    assert (err <= bound).all(), np.max(err - bound)
    assert np.array_equal(got[:, 2], depth[v, u])  # z is the depth itself
    # the ray slopes of the image corners, written out by hand
    corner = np.array([(0 - 17.75) / 61.25, (36 - 17.75) / 61.25, (0 - 9.5) / 47.5, (22 - 9.5) / 47.5])
    assert np.allclose(corner, [-0.289795918, 0.297959184, -0.2, 0.263157895], atol=1e-9)


def test_world_points_match_float64_transform():
    cam = _camera()
    w, _ = _world(cam)
    depth = _depth(cam, seed=4)
    _, got = oracle.observed(w, depth)
    exact_c, _, _ = _exact_camera_points(cam, depth)
    exact, S = _exact_world(cam, exact_c)
    err = np.abs(got.astype(np.float64) - exact)
    bound = 4 * 2.0 ** -23 * S * 1.001  # camera-point error through R, plus four roundings
    assert (err <= bound).all(), np.max(err - bound)
    assert err.max() < 2e-6  # metres: far below any sign or transpose slip


def test_table_plane_points_lie_on_the_plane():
    """A depth image of the bare table (z = 0) made by float64 ray-plane
    intersection: the observed world points lie on the plane, and at the
    (x, y) where each pixel's ray meets it."""
    cam = synth.camera_c2()
    w, _ = _world(cam)
    T = cam.T_wc.astype(np.float64)
    R, t = T[:, :3], T[:, 3]
    vv, uu = np.mgrid[0:cam.H, 0:cam.W]
    ray = np.stack([(uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy, np.ones_like(uu, np.float64)], -1)
    dirw = ray @ R.T
    s = -t[2] / dirw[..., 2]  # ray parameter = camera Z (the ray has z = 1 in the camera frame)
    depth = np.where(s > 0, s, 0.0).astype(np.float32)
    _, got = oracle.observed(w, depth)
    assert len(got) == cam.W * cam.H  # the camera looks down: every pixel sees the table
    assert np.abs(got[:, 2]).max() < 2e-6
    hit = (t[None, None, :] + s[..., None] * dirw).reshape(-1, 3)
    assert np.abs(got[:, :2].astype(np.float64) - hit[:, :2]).max() < 5e-6


def test_box_points_lie_on_its_faces():
    """Noise-free sensor depth of the C1 box at yaw 0 (the double-precision
    ray caster of the input generator, not the method's rasteriser): every
    observed world point lies on one of the box's face planes, inside that
    face."""
    c1 = synth.workload_c1()
    cam = c1.cam
    w = oracle.World.of(c1)
    o = synth.objs([(0, 4, 5, 0)])
    depth = synth.raycast_depth(cam, c1.meshes, c1.grid, o).astype(np.float32)
    _, q = oracle.observed(w, depth)
    assert len(q) > 150
    q = q.astype(np.float64)
    ox, oy = float(c1.grid.xs[4]), float(c1.grid.ys[5])
    lo = np.array(c1.meshes[0].verts, np.float64).min(0)
    hi = np.array(c1.meshes[0].verts, np.float64).max(0)
    lo[:2] += (ox, oy)
    hi[:2] += (ox, oy)
    tol = 1e-5
    inside = ((q >= lo - tol) & (q <= hi + tol)).all(1)
    on_face = np.zeros(len(q), bool)
    for k in range(3):
        on_face |= (np.abs(q[:, k] - lo[k]) <= tol) | (np.abs(q[:, k] - hi[k]) <= tol)
    assert inside.all() and on_face.all()
    # the camera sits at y = -1 looking down: it sees the top and the -y face
    assert (np.abs(q[:, 2] - hi[2]) <= tol).sum() > 20
    assert (np.abs(q[:, 1] - lo[1]) <= tol).sum() > 20


def test_volume_membership_uses_the_sensor_pose():
    """n_vol at the root = |I n V(O)| (Sec. III-A, Sec. IV-C), against an
    inscribed-cylinder test on world points computed here in float64 from
    (u, v, d) and T_world_cam; points within the binary32 bound of the
    cylinder's surface are not counted either way."""
    c1 = synth.workload_c1()
    w = oracle.World.of(c1)
    exact_c, _, _ = _exact_camera_points(c1.cam, c1.depth)
    q, S = _exact_world(c1.cam, exact_c)
    slack = 4 * 2.0 ** -23 * S.max() * 1.001 + 1e-7
    hyps = np.concatenate([c1.gt, synth.all_hypotheses(c1.grid, [0, 1])[::13]])
    recs = oracle.eval_batch(w, c1.depth, [c1.gt[:0]], np.zeros(len(hyps), np.int32), hyps, 2)
    checked = nonzero = 0
    for o, r in zip(hyps, recs):
        m = c1.meshes[int(o["mesh"])]
        x0, y0 = float(c1.grid.xs[o["ix"]]), float(c1.grid.ys[o["iy"]])
        rho = np.hypot(q[:, 0] - x0, q[:, 1] - y0)
        sure_in = (rho <= m.vol_r - 2 * slack) & (q[:, 2] >= m.vol_zlo + slack) & (q[:, 2] <= m.vol_zhi - slack)
        maybe_in = (rho <= m.vol_r + 2 * slack) & (q[:, 2] >= m.vol_zlo - slack) & (q[:, 2] <= m.vol_zhi + slack)
        assert sure_in.sum() <= r[6] <= maybe_in.sum(), (o, r[6], sure_in.sum(), maybe_in.sum())
        checked += sure_in.sum() == maybe_in.sum()
        nonzero += r[6] > 0
    assert checked > 0.9 * len(hyps) and nonzero >= 2


@pytest.mark.parametrize("flip", ["t", "R"])
def test_a_wrong_sensor_pose_moves_the_volume_counts(flip):
    """The counts above depend on the pose: with T_world_cam's translation
    negated or its rotation transposed, the same depth image gives other
    n_vol values (so the previous test would catch either slip)."""
    c1 = synth.workload_c1()
    T = c1.cam.T_wc.copy()
    if flip == "t":
        T[:, 3] = -T[:, 3]
    else:
        T[:, :3] = T[:, :3].T.copy()
    bad = synth.Camera(c1.cam.W, c1.cam.H, c1.cam.fx, c1.cam.fy, c1.cam.cx, c1.cam.cy, T)
    good_w, bad_w = oracle.World.of(c1), oracle.World(bad, c1.meshes, c1.grid, c1.delta)
    hyps = synth.all_hypotheses(c1.grid, [0, 1])[::13]
    hp = np.zeros(len(hyps), np.int32)
    recs_good = oracle.eval_batch(good_w, c1.depth, [c1.gt[:0]], hp, hyps, 2)
    recs_bad = oracle.eval_batch(bad_w, c1.depth, [c1.gt[:0]], hp, hyps, 2)
    assert recs_good[:, 6].sum() > 50 and not np.array_equal(recs_good[:, 6], recs_bad[:, 6])
