"""GPU parity of the ICP refinement (Sec. IV-E-1; Sec. V-B: correspondences
within 2 cm) through the C ABI against the CPU oracle.

Every record is compared in full and bit for bit: the motion's four doubles,
|M|, the pairs of the last matching, the fits made and the stop reason. The
arithmetic is fixed step by step (binary32 render, back-projection, motion
and distances; exact integer sums; one double fit in a fixed order), so the
two sides agree exactly or one of them is wrong.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1510_05613_gb300 import accuracy, perch, synth

pytestmark = pytest.mark.gpu

FIELDS = ("c", "s", "tx", "ty", "n_model", "n_corr", "iters", "status")


def _compare(got, exp, hyps=None):
    bad = [i for i in range(len(exp)) if any(got[f][i] != exp[f][i] for f in FIELDS)]
    assert not bad, (f"{len(bad)} of {len(exp)} records differ, first {bad[:3]}"
                     f"{'' if hyps is None else ' ' + str(hyps[bad[:3]])}: gpu {got[bad[:3]]} oracle {exp[bad[:3]]}")


@pytest.fixture(scope="module")
def c1():
    wl = synth.workload_c1()
    p = perch.Perch(0)
    p.setup(wl)
    return wl, p, oracle.World.of(wl)


@pytest.fixture(scope="module")
def off():
    wl = synth.workload_c2_off_grid(0)
    p = perch.Perch(0)
    p.setup(wl)
    return wl, p, oracle.World.of(wl)


def _near(grid, objs, allh, reach=2):
    """Hypotheses within `reach` grid cells of the objects (the ones whose
    model meets the cloud), every yaw."""
    keep = np.zeros(len(allh), bool)
    for o in objs:
        keep |= (np.abs(allh["ix"].astype(int) - int(o["ix"])) <= reach) & \
                (np.abs(allh["iy"].astype(int) - int(o["iy"])) <= reach)
    return allh[keep]


def test_icp_bit_exact_c1(c1):
    wl, p, w = c1
    allh = synth.all_hypotheses(wl.grid, [0, 1])
    hyps = np.concatenate([allh[::23], _near(wl.grid, wl.gt, allh, 1)[::3]])
    parents = [wl.gt[:0], wl.gt[:1], wl.gt[1:]]
    hp = (np.arange(len(hyps)) % 3).astype(np.int32)
    got = p.perch_icp_refine(parents, hp, hyps, 0.02, 20)
    exp = oracle.icp_refine(w, wl.depth, parents, hp, hyps, 0.02, 20)
    _compare(got, exp, hyps)
    # the batch spans every way the iteration stops
    assert {oracle.ICP_FEW, oracle.ICP_CONVERGED, oracle.ICP_CAP} <= set(exp["status"].tolist())
    assert (exp["n_corr"] > 100).sum() > 10


@pytest.mark.parametrize("radius,max_iter", [(0.0, 5), (0.005, 1), (0.03, 0), (0.05, 7)])
def test_icp_bit_exact_c1_radii_and_limits(c1, radius, max_iter):
    wl, p, w = c1
    allh = synth.all_hypotheses(wl.grid, [0, 1])
    hyps = _near(wl.grid, wl.gt, allh, 1)[::5]
    parents = [wl.gt[:0], wl.gt[:1]]
    hp = (np.arange(len(hyps)) % 2).astype(np.int32)
    got = p.perch_icp_refine(parents, hp, hyps, radius, max_iter)
    exp = oracle.icp_refine(w, wl.depth, parents, hp, hyps, radius, max_iter)
    _compare(got, exp, hyps)


def test_icp_bit_exact_off_grid_c2_and_accuracy(off):
    """640 x 480: each object of the off-grid scene against the objects
    before it (the refinement of the successors on the path to the true
    scene), plus neighbouring grid poses; then the refined poses against the
    ground truth."""
    wl, p, w = off
    allh = synth.all_hypotheses(wl.grid, [0, 1, 2])
    near = _near(wl.grid, wl.gt, allh, 1)
    rng = np.random.default_rng(3)
    extra = near[rng.choice(len(near), 21, replace=False)]
    objs = wl.gt
    parents = [objs[:k] for k in range(len(objs))]
    hyps = np.concatenate([objs, extra])
    hp = np.concatenate([np.arange(len(objs)), rng.integers(0, len(objs), len(extra))]).astype(np.int32)
    got = p.perch_icp_refine(parents, hp, hyps, 0.02, 20)
    exp = oracle.icp_refine(w, wl.depth, parents, hp, hyps, 0.02, 20)
    _compare(got, exp, hyps)
    truth = accuracy.true_poses(wl)
    for k, o in enumerate(objs):
        _, x, y, _ = perch.refined_pose(wl.grid, o, got[k])
        gx, gy = float(wl.grid.xs[o["ix"]]), float(wl.grid.ys[o["iy"]])
        before = math.hypot(gx - truth[k][1], gy - truth[k][2])
        after = math.hypot(x - truth[k][1], y - truth[k][2])
        assert after < 2e-3 and after < 0.25 * before, (k, before, after)


def test_refine_scene_against_the_other_objects(off):
    wl, p, w = off
    recs, poses = p.perch_refine_scene(wl.gt[::-1])
    objs = wl.gt[::-1]
    others = [np.concatenate([objs[:k], objs[k + 1:]]) for k in range(len(objs))]
    exp = oracle.icp_refine(w, wl.depth, others, np.arange(len(objs)), objs, 0.02, 20)
    _compare(recs, exp)
    assert [q[0] for q in poses] == [int(o["mesh"]) for o in objs]


def test_icp_full_size_sampled(off):
    """The full root expansion of the 640 x 480 grid (3 meshes x 50 x 50 x 16
    poses, every successor refined as the paper does) in one launch; a
    sample, weighted to the successors that meet the cloud, against the
    oracle one by one."""
    wl, p, w = off
    hyps = synth.all_hypotheses(wl.grid, [0, 1, 2])
    hp = np.zeros(len(hyps), np.int32)
    got = p.perch_icp_refine([wl.gt[:0]], hp, hyps, 0.02, 20)
    active = np.nonzero(got["n_corr"] >= 3)[0]
    rng = np.random.default_rng(4)
    pick = np.concatenate([rng.choice(active, 12, replace=False), rng.choice(len(hyps), 4, replace=False)])
    exp = oracle.icp_refine(w, wl.depth, [wl.gt[:0]], hp[pick], hyps[pick], 0.02, 20)
    _compare(got[pick], exp, hyps[pick])
    # properties at any size: a unit turn, |M| >= pairs, fits <= 20
    assert np.allclose(got["c"] ** 2 + got["s"] ** 2, 1.0, atol=1e-12)
    assert np.all(got["n_corr"] <= got["n_model"]) and np.all(got["iters"] <= 20)
    assert np.all(got["status"] <= 3)


def test_icp_edge_cases(c1):
    wl, p, w = c1
    hyps = np.concatenate([wl.gt, synth.objs([(0, 0, 0, 0), (1, 9, 9, 7)])])
    hp = np.zeros(len(hyps), np.int32)
    # max_iter 0: the identity, nothing matched
    got = p.perch_icp_refine([wl.gt[:0]], hp, hyps, 0.02, 0)
    assert np.all(got["c"] == 1.0) and np.all(got["s"] == 0.0) and np.all(got["status"] == perch.PERCH_ICP_CAP)
    _compare(got, oracle.icp_refine(w, wl.depth, [wl.gt[:0]], hp, hyps, 0.02, 0))
    # an object at the very pose of a parent object adds no pixel in front of it
    got = p.perch_icp_refine([wl.gt], np.zeros(1, np.int32), wl.gt[:1], 0.02, 20)
    assert got["n_model"][0] == 0 and got["status"][0] == perch.PERCH_ICP_FEW
    # empty input
    assert len(p.perch_icp_refine([wl.gt[:0]], np.zeros(0, np.int32), wl.gt[:0], 0.02, 20)) == 0
    # arguments the host rejects
    for args in ((0.02, -1), (0.02, 1001), (-0.01, 20), (float("nan"), 20), (2.0, 20)):
        with pytest.raises(perch.PerchError) as e:
            p.perch_icp_refine([wl.gt[:0]], hp, hyps, *args)
        assert e.value.code == perch.PERCH_E_ARG
    with pytest.raises(perch.PerchError):
        p.perch_icp_refine([wl.gt[:0]], np.array([1], np.int32), hyps[:1], 0.02, 20)


def test_icp_dev_path_flags_bad_indices(c1):
    import torch
    wl, p, w = c1
    hyps = np.concatenate([wl.gt, wl.gt])
    P, plen, stride = p.pack_parents([wl.gt[:0], wl.gt[:1]])
    hp = np.array([0, 1, 2, -1], np.int32)  # the last two name no parent
    dev = torch.device("cuda:0")
    Pt = torch.from_numpy(P.view(np.int16).copy()).to(dev)
    plt = torch.from_numpy(plen).to(dev)
    hpt = torch.from_numpy(hp).to(dev)
    ht = torch.from_numpy(hyps.view(np.int16).copy()).to(dev)
    out = torch.zeros(len(hyps) * 48, dtype=torch.uint8, device=dev)
    p.perch_icp_refine_dev(Pt, stride, plt, hpt, ht, 0.02, 20, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(perch.ICP)
    assert np.all(got["status"][2:] == perch.FLAG_BAD_INDEX)
    exp = oracle.icp_refine(w, wl.depth, [wl.gt[:0], wl.gt[:1]], hp[:2], hyps[:2], 0.02, 20)
    _compare(got[:2], exp)


def test_icp_follows_a_new_observation():
    """The cloud's grid is rebuilt when the observation changes."""
    wl0, wl1 = synth.workload_c1(0), synth.workload_c1(1)
    p = perch.Perch(0)
    p.setup(wl0)
    hyps = np.concatenate([wl0.gt, wl1.gt])
    hp = np.zeros(len(hyps), np.int32)
    p.perch_icp_refine([wl0.gt[:0]], hp, hyps, 0.02, 20)
    p.perch_set_observation(wl1.depth, wl1.cam.fxfycxcy, wl1.cam.T_wc, wl1.delta)
    got = p.perch_icp_refine([wl1.gt[:0]], hp, hyps, 0.02, 20)
    _compare(got, oracle.icp_refine(oracle.World.of(wl1), wl1.depth, [wl1.gt[:0]], hp, hyps, 0.02, 20))
    p.close()
