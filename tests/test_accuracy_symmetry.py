"""Pose accuracy (Sec. V-D's criterion) and the search over rotationally
symmetric meshes (Sec. IV-E: a symmetric object needs only (x, y)).

The accuracy report is checked on hand-made poses: the strict thresholds of
the criterion, the shortest angular difference, the symmetry period, and the
pairing of same-type objects. The symmetric tree is pinned by enumeration:
uniform-cost search over it equals the exhaustive minimum over all ordered
placements at the kept yaws, and the kept yaws are the ones the meshes'
vertex sets make equivalent.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import search
from paper_1510_05613_gb300 import accuracy, synth


def test_angular_difference_shortest_and_modulo_symmetry():
    d = math.radians
    assert accuracy.angular_difference(d(170), d(-175), 1) == pytest.approx(d(15))
    assert accuracy.angular_difference(d(10), d(350), 1) == pytest.approx(d(20))
    assert accuracy.angular_difference(0.0, d(90), 4) == pytest.approx(0.0, abs=1e-12)
    assert accuracy.angular_difference(0.0, d(100), 4) == pytest.approx(d(10))
    assert accuracy.angular_difference(d(5), d(185), 2) == pytest.approx(0.0, abs=1e-12)
    assert accuracy.angular_difference(d(1), d(359), 128) == pytest.approx(d(358 - 127 * 360 / 128))


def test_pose_errors_pair_same_type_objects_and_count_strictly():
    grid = synth.pose_grid(0.0, 0.1, 5, 8)
    pred = synth.objs([(0, 1, 1, 0), (0, 3, 3, 2), (1, 2, 2, 1)])
    truth = [(0, 0.3, 0.3 + 0.004, math.radians(90 + 3)),  # the second box, 4 mm and 3 deg away
             (0, 0.1, 0.1, 0.0),                             # the first box, exact
             (1, 0.2 + 0.0105, 0.2, math.radians(45 + 50))]  # the cylinder, 1.05 cm away, 50 deg
    errs = accuracy.pose_errors(pred, truth, grid, syms=[2, 1])
    assert [e[0] for e in errs] == [0, 0, 1]
    by = sorted(errs)
    assert by[0][1] == pytest.approx(0.0, abs=1e-7) and by[0][2] == pytest.approx(0.0, abs=1e-5)
    assert by[1][1] == pytest.approx(0.004, abs=1e-7) and by[1][2] == pytest.approx(3.0, abs=1e-4)
    cnt = accuracy.correct_counts(errs, dts=(0.005, 0.01, 0.011), dthetas=(5.0, 60.0))
    assert cnt[(0.005, 5.0)] == 2 and cnt[(0.01, 60.0)] == 2
    assert cnt[(0.011, 60.0)] == 3 and cnt[(0.011, 5.0)] == 2
    # a type with no prediction is wrong at every threshold
    errs2 = accuracy.pose_errors(pred[:1], truth, grid, syms=[2, 1])
    assert sum(1 for e in errs2 if math.isinf(e[1])) == 2


def test_true_poses_add_the_off_grid_offsets():
    wl = synth.workloads_c5(1, grid=synth.pose_grid(-0.48, 0.04, 25, 8), k_range=(3, 3), off_grid=1.0)[0]
    tp = accuracy.true_poses(wl)
    for (m, x, y, yaw), o, j in zip(tp, wl.gt, wl.extra["jitter"]):
        assert x == pytest.approx(float(wl.grid.xs[o["ix"]]) + j[0])
        assert y == pytest.approx(float(wl.grid.ys[o["iy"]]) + j[1])


def test_symmetric_yaws_follow_the_vertex_sets():
    """A kept yaw class is exactly the set of yaws whose turned vertex sets
    coincide (to float32 rounding of the vertices)."""
    grid = synth.pose_grid(-0.49, 0.02, 50, 16)
    meshes = synth.meshes_c2()
    keep = search.symmetric_yaws(grid, [m.sym for m in meshes])
    assert [len(keep[m]) for m in range(3)] == [8, 1, 4]
    th = [math.atan2(float(s), float(c)) for c, s in grid.cos_sin]
    for m, mesh in enumerate(meshes):
        v = mesh.verts.astype(np.float64)
        for k in range(16):
            same = []
            for j in keep[m]:
                a = th[k] - th[j]
                r = np.stack([math.cos(a) * v[:, 0] - math.sin(a) * v[:, 1],
                              math.sin(a) * v[:, 0] + math.cos(a) * v[:, 1]], 1)
                # every turned vertex lands on a vertex (brute force over a sample)
                d = np.sqrt(((r[:200, None, :] - v[None, :, :2]) ** 2).sum(-1)).min(1)
                same.append(d.max() < 1e-6)
            assert sum(same) == 1, (mesh.name, k, same)  # exactly one kept yaw represents yaw k


def test_symmetric_tree_search_equals_its_exhaustive_minimum():
    """Uniform-cost search over the tree with the symmetric meshes' other
    yaws removed returns the minimum over all ordered placements at the kept
    yaws (brute force on a 4 x 4 x 4 grid)."""
    grid = synth.pose_grid(-0.15, 0.1, 4, 4)
    wl = synth.workload_c1(scene=3, grid=grid)
    w = oracle.World.of(wl)
    yaws = search.symmetric_yaws(grid, [m.sym for m in wl.meshes])
    assert [len(yaws[0]), len(yaws[1])] == [2, 1]
    cost, key, _ = search.uniform_cost_search(w, wl.depth, grid, wl.mesh_multiset, yaws=yaws)
    hyps = search._children(grid, [0, 1], yaws)
    h0, h1 = hyps[hyps["mesh"] == 0], hyps[hyps["mesh"] == 1]
    best = None
    for first, second in ((h0, h1), (h1, h0)):
        r1 = oracle.eval_batch(w, wl.depth, [first[:0]], np.zeros(len(first), np.int32), first, 2)
        for i, a in enumerate(first):
            if r1[i, 3] > 0:
                continue
            r2 = oracle.eval_batch(w, wl.depth, [first[i:i + 1]], np.zeros(len(second), np.int32), second, 2)
            for j, b in enumerate(second):
                if r2[j, 3] > 0:
                    continue
                c = int(r1[i, :3].sum() + r2[j, :3].sum())
                k = search.key_of([a, b])
                if best is None or (c, k) < best:
                    best = (c, k)
    assert (cost, key) == best
