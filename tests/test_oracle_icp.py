"""Pins of the oracle's ICP refinement (Sec. IV-E-1: each newly rendered
object's non-occluded portion is aligned with the observed cloud; Sec. V-B:
correspondences only within 2 cm).

Each part is pinned to something outside the oracle:
  - the closed-form fit against motions the test makes itself (a point set
    turned and shifted in float64) and against an SVD (Kabsch) fit of the
    same pairs in float64, a different method for the same optimum; a
    transposed rotation, a sign error or a wrong centroid fails them;
  - the correspondence rule against a float64 brute-force nearest-neighbour
    search over the observed cloud (scipy's k-d tree as a second one);
  - the model set against the edge cost's |dR| (n_new) of the same successor,
    computed by the oracle's edge-cost code;
  - the whole iteration against exact closed forms (an observation that is
    the object's own render gives the identity after one fit, exactly) and
    against ground truth: an object observed off the grid by the ray-cast
    sensor (an independent renderer) is brought back to its true pose.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1510_05613_gb300 import synth


def _rot(th):
    return np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])


def _kabsch2(m, q):
    """Best planar turn and shift of m onto q (float64, SVD)."""
    mc, qc = m[:, :2].mean(0), q[:, :2].mean(0)
    H = (m[:, :2] - mc).T @ (q[:, :2] - qc)
    U, _, Vt = np.linalg.svd(H)
    D = np.diag([1.0, np.sign(np.linalg.det(Vt.T @ U.T))])
    R = Vt.T @ D @ U.T
    return R, qc - R @ mc


@pytest.mark.parametrize("th,t", [(0.0, (0.0, 0.0)), (0.1, (0.01, -0.02)), (-0.35, (0.004, 0.0)),
                                  (2.5, (-0.3, 0.2)), (-3.0, (1.5, -2.0)), (math.pi / 2, (0.0, 0.5))])
def test_fit_recovers_a_known_motion(th, t):
    rng = np.random.default_rng(5)
    m = np.column_stack([rng.uniform(-0.08, 0.08, 400) + 0.3, rng.uniform(-0.05, 0.05, 400) - 0.2,
                         rng.uniform(0.0, 0.15, 400)]).astype(np.float32)
    q = m.astype(np.float64).copy()
    q[:, :2] = m[:, :2].astype(np.float64) @ _rot(th).T + np.array(t)
    q[:, 2] += rng.normal(0, 0.01, 400)  # heights do not enter the planar fit
    (c, s, tx, ty), st = oracle.icp_fit(m, q.astype(np.float32))
    assert st == 0
    # fixed point of 2^-16 m on ~0.1 m of spread: a few 1e-5 in the angle
    assert abs(c - math.cos(th)) < 5e-5 and abs(s - math.sin(th)) < 5e-5
    assert abs(c * c + s * s - 1.0) < 1e-12
    assert abs(tx - t[0]) < 1e-4 * (1 + abs(t[0])) and abs(ty - t[1]) < 1e-4 * (1 + abs(t[1]))


def test_fit_matches_svd_on_noisy_pairs():
    rng = np.random.default_rng(6)
    for trial in range(20):
        n = int(rng.integers(3, 3000))
        m = rng.normal(0, 0.05, (n, 3)).astype(np.float32)
        m[:, 0] += np.float32(rng.uniform(-0.5, 0.5))
        q = m.astype(np.float64).copy()
        th = rng.uniform(-math.pi, math.pi)
        q[:, :2] = q[:, :2] @ _rot(th).T + rng.uniform(-0.1, 0.1, 2)
        q += rng.normal(0, 0.003, q.shape)
        q = q.astype(np.float32)
        (c, s, tx, ty), st = oracle.icp_fit(m, q)
        assert st == 0
        R, tt = _kabsch2(m.astype(np.float64), q.astype(np.float64))
        # rounding to 2^-16 m moves each coordinate by a uniform error of
        # sd 2^-16 / sqrt(12) = 4.4e-6 m; the angle then moves by about
        # sd sqrt(2) / (sqrt(n) rms radius): allow 5 of those
        rms = float(np.sqrt(((m[:, :2] - m[:, :2].mean(0)) ** 2).sum(1).mean()))
        tol = 5 * 4.4e-6 * math.sqrt(2) / (math.sqrt(n) * rms)
        assert abs(c - R[0, 0]) < tol and abs(s - R[1, 0]) < tol, (trial, c - R[0, 0], tol)
        cen = float(np.abs(m[:, :2].mean(0)).max())
        assert np.allclose([tx, ty], tt, atol=5 * 4.4e-6 + tol * cen), trial


def test_fit_degenerate_and_too_few_pairs():
    p = np.array([[0.1, 0.2, 0.0]] * 5, np.float32)
    assert oracle.icp_fit(p, p)[1] == 1  # every pair at one point: no turn is defined
    m = np.array([[0.0, 0.0, 0.0], [0.1, 0.0, 0.0]], np.float32)
    assert oracle.icp_fit(m, m)[1] == 2  # fewer than 3 pairs
    far = np.array([[40.0, 0.0, 0.0], [40.1, 0.0, 0.0], [40.0, 0.1, 0.0]], np.float32)
    assert oracle.icp_fit(far, far)[1] == 2  # pairs beyond 32 m are left out
    assert oracle.icp_fit(far[:, [1, 0, 2]], far[:, [1, 0, 2]])[1] == 2  # in y as well
    near = far - np.float32([39.9, 0.0, 0.0])
    assert oracle.icp_fit(near, near)[1] == 0


def test_fit_identity_is_exact():
    rng = np.random.default_rng(7)
    m = rng.normal(0, 0.05, (100, 3)).astype(np.float32)
    assert oracle.icp_fit(m, m) == ((1.0, 0.0, 0.0, 0.0), 0)


def _c1_scene():
    wl = synth.workload_c1()
    return wl, oracle.World.of(wl)


def test_correspondences_match_brute_force():
    wl, w = _c1_scene()
    _, Iw = oracle.observed(w, wl.depth)
    rng = np.random.default_rng(8)
    base = Iw[rng.choice(len(Iw), 300)].astype(np.float64)
    P = np.concatenate([base + rng.uniform(-0.03, 0.03, base.shape), rng.uniform(-0.3, 0.3, (100, 3))])
    P = P.astype(np.float32)
    r = 0.02
    idx = oracle.icp_match(w, wl.depth, P, r)
    d = np.sqrt(((P[:, None, :].astype(np.float64) - Iw[None, :, :].astype(np.float64)) ** 2).sum(-1))
    dmin, amin = d.min(1), d.argmin(1)
    tree = pytest.importorskip("scipy.spatial").cKDTree(Iw.astype(np.float64))
    kd, _ = tree.query(P.astype(np.float64))
    assert np.allclose(kd, dmin, atol=1e-12)
    n_matched = 0
    for k in range(len(P)):
        if dmin[k] > r * (1 + 1e-5):
            assert idx[k] == -1, k
        elif dmin[k] < r * (1 - 1e-5):
            assert idx[k] >= 0, k
            assert d[k, idx[k]] <= dmin[k] + 1e-6, k  # the nearest, up to binary32 rounding of d^2
            n_matched += 1
            if np.sort(d[k])[1] > dmin[k] + 1e-6:  # a clear winner: the very same point
                assert idx[k] == amin[k], k
    assert n_matched > 200


def test_model_set_is_the_new_objects_dR():
    """|M| = n_new of the edge cost for valid successors: the object's pixels
    in front of the parent are exactly those where the parent is empty."""
    wl, w = _c1_scene()
    allh = synth.all_hypotheses(wl.grid, [0, 1])
    g0 = wl.gt[0]
    # in front of the parent's object (the camera looks along +y): many
    # of these occlude it and break Eq. (3)
    front = allh[(np.abs(allh["ix"].astype(int) - int(g0["ix"])) <= 2) & (allh["iy"] < g0["iy"]) &
                 (allh["iy"] >= int(g0["iy"]) - 3)][::3]
    sample = allh[::37]
    hyps = np.concatenate([sample, front])
    parents = [wl.gt[:0], wl.gt[:1]]
    hp = np.concatenate([np.arange(len(sample)) % 2, np.ones(len(front))]).astype(np.int32)
    rec = oracle.eval_batch(w, wl.depth, parents, hp, hyps, wl.K)
    icp = oracle.icp_refine(w, wl.depth, parents, hp, hyps, 0.02, 0)
    valid = rec[:, 3] == 0
    assert valid.sum() > 20 and (~valid).sum() > 0
    assert np.array_equal(icp["n_model"][valid], rec[valid, 4])
    assert np.all(icp["n_model"][~valid] > rec[~valid, 4])  # plus the pixels in front of the parent
    assert np.all(icp["iters"] == 0) and np.all(icp["status"] == oracle.ICP_CAP)
    assert np.all(icp["c"] == 1.0) and np.all(icp["s"] == 0.0)


def _object_scene(jitter=None, sigma=0.0, dropout=0.0, iyaw=3, seed=1):
    cam = synth.camera_c2()
    meshes = [synth.box_mesh(0.10, 0.06, 0.15, 29)]
    grid = synth.pose_grid(-0.49, 0.02, 50, 16)
    gt = synth.objs([(0, 25, 25, iyaw)])
    depth = synth.observe(cam, meshes, grid, gt, sigma, dropout, seed, jitter=None if jitter is None else [jitter])
    return oracle.World(cam, meshes, grid, 0.01), grid, gt, depth


def test_own_render_gives_the_identity_exactly():
    w, grid, gt, _ = _object_scene()
    z, _ = oracle.render(w, gt)
    depth = np.where(np.isfinite(z), z, 0.0).astype(np.float32)
    rec = oracle.icp_refine(w, depth, [gt[:0]], [0], gt, 0.02, 20)[0]
    # every model point meets itself (d = 0): the fit of identical sums is
    # exactly the identity, and the second matching repeats the first
    assert (rec["c"], rec["s"], rec["tx"], rec["ty"]) == (1.0, 0.0, 0.0, 0.0)
    assert rec["iters"] == 1 and rec["status"] == oracle.ICP_CONVERGED
    assert rec["n_corr"] == rec["n_model"] == int(np.isfinite(z).sum())


def test_empty_observation_and_zero_radius():
    w, grid, gt, depth = _object_scene()
    rec = oracle.icp_refine(w, np.zeros_like(depth), [gt[:0]], [0], gt, 0.02, 20)[0]
    assert rec["status"] == oracle.ICP_FEW and rec["iters"] == 0 and rec["n_corr"] == 0
    assert (rec["c"], rec["s"], rec["tx"], rec["ty"]) == (1.0, 0.0, 0.0, 0.0)
    # r = 0 keeps only exact coincidences: none under sensor noise
    w, grid, gt, depth = _object_scene(sigma=0.003, seed=2)
    rec = oracle.icp_refine(w, depth, [gt[:0]], [0], gt, 0.0, 20)[0]
    assert rec["status"] == oracle.ICP_FEW and rec["n_corr"] == 0


@pytest.mark.parametrize("jit", [(0.008, -0.006, 5.0), (-0.009, 0.009, -10.0), (0.005, 0.007, 8.0)])
def test_off_grid_object_is_brought_to_its_true_pose(jit):
    dx, dy, dyaw = jit[0], jit[1], math.radians(jit[2])
    w, grid, gt, depth = _object_scene((dx, dy, dyaw))
    rec = oracle.icp_refine(w, depth, [gt[:0]], [0], gt, 0.02, 20)[0]
    x, y, yaw = oracle.icp_pose(grid, gt[0], rec)
    o = gt[0]
    tx, ty = float(grid.xs[o["ix"]]) + dx, float(grid.ys[o["iy"]]) + dy
    tyaw = math.atan2(float(grid.cos_sin[o["iyaw"], 1]), float(grid.cos_sin[o["iyaw"], 0])) + dyaw
    assert math.hypot(x - tx, y - ty) < 1e-3  # from ~1 cm off to under 1 mm
    assert abs(math.degrees(yaw - tyaw)) < 1.0  # from 5-10 degrees off to under 1
    assert rec["n_corr"] > 0.9 * rec["n_model"]


def test_noisy_observation_still_converges_near_the_truth():
    jit = (0.007, 0.004, math.radians(-6.0))
    w, grid, gt, depth = _object_scene(jit, sigma=0.003, dropout=0.05, seed=4)
    rec = oracle.icp_refine(w, depth, [gt[:0]], [0], gt, 0.02, 20)[0]
    x, y, yaw = oracle.icp_pose(grid, gt[0], rec)
    o = gt[0]
    tx, ty = float(grid.xs[o["ix"]]) + jit[0], float(grid.ys[o["iy"]]) + jit[1]
    assert math.hypot(x - tx, y - ty) < 3e-3


def test_refined_pose_of_binding_and_oracle_agree():
    """The binding's pose arithmetic (perch.refined_pose) and the oracle's
    (icp_pose) move a grid pose by a record's motion the same way; a pure
    shift moves (x, y) only, a turn about the origin turns (x, y) and the yaw."""
    from paper_1510_05613_gb300 import perch
    grid = synth.pose_grid(-0.49, 0.02, 50, 16)
    o = synth.objs([(0, 30, 10, 5)])[0]
    for c, s, tx, ty in [(1.0, 0.0, 0.01, -0.02), (math.cos(0.3), math.sin(0.3), 0.0, 0.0),
                         (math.cos(-1.2), math.sin(-1.2), 0.004, 0.003)]:
        rec = np.zeros(1, perch.ICP)[0]
        rec["c"], rec["s"], rec["tx"], rec["ty"] = c, s, tx, ty
        _, x, y, yaw = perch.refined_pose(grid, o, rec)
        assert np.allclose((x, y, yaw), oracle.icp_pose(grid, o, rec), atol=1e-15)
        x0, y0 = float(grid.xs[o["ix"]]), float(grid.ys[o["iy"]])
        assert np.allclose((x, y), (c * x0 - s * y0 + tx, s * x0 + c * y0 + ty))
        th0 = math.atan2(float(grid.cos_sin[o["iyaw"], 1]), float(grid.cos_sin[o["iyaw"], 0]))
        assert abs(yaw - th0 - math.atan2(s, c)) < 1e-12
