"""Pins of the oracle's tree search (MSGT of Sec. IV-A, search of Sec. IV-B).

Uniform-cost search (A* with the trivial admissible heuristic h0 = 0 that the
paper uses as its anchor heuristic) must return the exhaustive minimum over
every valid ordered sequence of placements, the brute force of Sec. III-B
restricted to monotone orders.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import search
from paper_1510_05613_gb300 import synth


@pytest.fixture(scope="module")
def small_c1():
    # C1 camera and meshes on a reduced 4 x 4 x 4 pose grid (64 poses/object)
    grid = synth.pose_grid(-0.15, 0.1, 4, 4)
    return synth.workload_c1(scene=3, grid=grid)


def test_uniform_cost_search_equals_exhaustive(small_c1):
    wl = small_c1
    w = oracle.World.of(wl)
    ex_cost, ex_key = search.exhaustive(w, wl.depth, wl.grid, wl.mesh_multiset)
    ucs_cost, ucs_key, expansions = search.uniform_cost_search(w, wl.depth, wl.grid, wl.mesh_multiset)
    assert ex_cost is not None
    assert (ucs_cost, ucs_key) == (ex_cost, ex_key)
    assert expansions >= 1


def test_exhaustive_on_three_objects_tiny_grid():
    grid = synth.pose_grid(-0.1, 0.1, 3, 2)
    cam, meshes = synth.camera_c1(), synth.meshes_c1()
    gt = synth.objs([(0, 0, 2, 0), (1, 2, 2, 1), (1, 1, 0, 0)])
    depth = synth.observe(cam, meshes, grid, gt, 0.002, 0.05, 77)
    w = oracle.World(cam, meshes, grid, 0.01)
    ms = [0, 1, 1]
    ex = search.exhaustive(w, depth, grid, ms)
    ucs = search.uniform_cost_search(w, depth, grid, ms)
    assert ex[0] is not None and (ucs[0], ucs[1]) == ex


def test_set_key_cost_is_order_independent(small_c1):
    """Every valid order of the same objects gives the same path cost (the
    reason the paper keeps a tree rather than a DAG)."""
    wl = small_c1
    w = oracle.World.of(wl)
    rng = np.random.default_rng(2)
    hyps = synth.all_hypotheses(wl.grid, [0, 1])
    n_multi = 0
    for _ in range(40):
        a = hyps[rng.integers(0, len(hyps) // 2)]
        b = hyps[len(hyps) // 2 + rng.integers(0, len(hyps) // 2)]
        costs = []
        for order in ([a, b], [b, a]):
            order = np.array(order, synth.OBJ_DTYPE)
            r0 = oracle.eval_batch(w, wl.depth, [order[:0]], np.zeros(1, np.int32), order[:1], 2)[0]
            r1 = oracle.eval_batch(w, wl.depth, [order[:1]], np.zeros(1, np.int32), order[1:], 2)[0]
            if r0[3] == 0 and r1[3] == 0:
                costs.append(int(r0[:3].sum() + r1[:3].sum()))
        if len(costs) == 2:
            n_multi += 1
            assert costs[0] == costs[1]
    assert n_multi > 5


@pytest.mark.parametrize("w", [1.0, 1.5, 3.0])
def test_focal_mha_respects_the_suboptimality_bound(small_c1, w):
    """Theorem 2: the returned cost is at most w times the optimum
    (exhaustive enumeration); Theorem 1: a solution is found; w = 1 is
    optimal."""
    wl = small_c1
    wo = oracle.World.of(wl)
    opt, opt_key = search.exhaustive(wo, wl.depth, wl.grid, wl.mesh_multiset)
    n_obs = oracle.observed(wo, wl.depth)[0].shape[0]
    cost, key, exp = search.focal_mha(wo, wl.depth, wl.grid, wl.mesh_multiset, w, n_obs=n_obs)
    assert cost is not None and opt <= cost <= w * opt + 1e-9
    if w == 1.0:
        assert cost == opt


def test_focal_mha_bound_holds_for_any_inadmissible_heuristic(small_c1):
    """Theorem 2 does not depend on what the inadmissible queues compute:
    with adversarial heuristics (preferring the emptiest states, or an
    arbitrary hash of the key) the answer still costs at most w * OPT."""
    wl = small_c1
    wo = oracle.World.of(wl)
    opt, _ = search.exhaustive(wo, wl.depth, wl.grid, wl.mesh_multiset)
    adversarial = lambda k: len(k)  # shallowest first
    scrambled = lambda k: hash(k) % 97
    for w in (1.0, 2.0):
        cost, key, exp = search.focal_mha(wo, wl.depth, wl.grid, wl.mesh_multiset, w,
                                          heuristics=(adversarial, scrambled))
        assert cost is not None and opt <= cost <= w * opt
        if w == 1.0:
            assert cost == opt
