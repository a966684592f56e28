"""The learned heuristic end to end on the GPU: training data from the exact
evaluator, training with the library's kernels, and Focal-MHA* with the
learned queue (heuristics bit 2: ordered by g + h_cnn across depths; bit 3:
the depth-first variant). Whatever the network predicts, the search must keep
Theorem 2's bound (cost <= w * OPT, OPT from uniform-cost search) and return
a scene whose cost is the exact sum of edge costs along one valid order of
its objects."""
import itertools

import numpy as np
import pytest
import torch

from paper_1510_05613_gb300 import heuristic as H
from paper_1510_05613_gb300 import perch, synth

pytestmark = pytest.mark.gpu

GRID = synth.pose_grid(-0.48, 0.04, 25, 8)


@pytest.fixture(scope="module")
def setup():
    # objects on the grid: small optimal costs, so plain search finishes quickly
    train_sc = H.training_scenes(24, grid=GRID, k_range=(2, 3), off_grid=0.0)
    test_sc = H.test_scenes(2, grid=GRID, K=3, off_grid=0.0)
    p = perch.Perch(0)
    tr = H.setup_scenes(p, train_sc)
    te = H.setup_scenes(p, test_sc, first_id=len(train_sc))
    stream = torch.cuda.Stream()
    n_onehot = len(train_sc[0].meshes) * GRID.n_yaw
    data, stats = H.make_dataset(p, train_sc, tr, per_parent=2048, seed=1)
    val, _ = H.make_dataset(p, test_sc, te, per_parent=512, seed=2)
    net = H.new_network(n_onehot, 256, seed=3, stream=stream)
    before = H.evaluate(net, val)
    losses, _ = H.train(net, data, epochs=4, batch=256, lr=1e-3, stream=stream)
    return p, net, test_sc, te, stats, losses, before, H.evaluate(net, val)


def test_training_learns_the_edge_cost(setup):
    p, net, test_sc, te, stats, losses, before, after = setup
    assert stats["pairs"] > 50000
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:20])
    assert after["mse"] < 0.5 * before["mse"]
    assert after["pearson"] > 0.4, after


def _path_cost(p, scene_id, K, objs):
    """Exact edge costs summed along every valid order of objs (Eq. (3))."""
    out = []
    for perm in itertools.permutations(range(len(objs))):
        o = objs[list(perm)]
        c, ok = 0, True
        for j in range(len(o)):
            r = perch.records(p.perch_eval_successors_multi([o[:j]], [scene_id], [K], np.zeros(1, np.int32),
                                                            o[j:j + 1]))[0]
            ok &= r[3] == 0
            c += int(r[:3].sum())
        if ok:
            out.append(c)
    return out


@pytest.mark.parametrize("w,heur", [(1.0, 7), (2.0, 7), (2.0, 4), (2.0, 9), (2.0, 8)])
def test_learned_queue_keeps_the_bound_and_exact_costs(setup, w, heur):
    p, net, test_sc, te, *_ = setup
    ms = [wl.mesh_multiset for wl in test_sc]
    p.perch_set_heuristic_net(net, 8)
    opt = p.perch_search_multi(te, ms, batch_states=2, w=1.0, heuristics=0)
    got = p.perch_search_multi(te, ms, batch_states=2, w=w, heuristics=heur)
    for o, g, sid, wl in zip(opt, got, te, test_sc):
        assert o["proven_optimal"] and o["cost"] >= 0
        assert o["cost"] <= g["cost"] <= w * o["cost"] + 1e-9
        if w == 1.0:  # optimal; among equal-cost goals either may be returned
            assert g["cost"] == o["cost"]
        # the returned scene was found before the search ended
        assert 0 < g["found_expansions"] <= g["expansions"] and g["found_seconds"] <= g["seconds"]
        costs = _path_cost(p, sid, wl.K, g["objs"])
        assert costs and min(costs) <= g["cost"] and g["cost"] in costs


def test_learned_bits_exclude_each_other(setup):
    p, net, test_sc, te, *_ = setup
    p.perch_set_heuristic_net(net, 8)
    with pytest.raises(perch.PerchError) as e:
        p.perch_search_multi(te[:1], [test_sc[0].mesh_multiset], w=2.0, heuristics=12)
    assert e.value.code == perch.PERCH_E_ARG


def test_learned_queue_needs_a_network(setup):
    p, net, test_sc, te, *_ = setup
    p.perch_set_heuristic_net(None, 8)
    with pytest.raises(perch.PerchError) as e:
        p.perch_search_multi(te[:1], [test_sc[0].mesh_multiset], w=2.0, heuristics=4)
    assert e.value.code == perch.PERCH_E_STATE
    p.perch_set_heuristic_net(net, 8)


def test_search_statistics_account_for_the_learned_queue(setup):
    p, net, test_sc, te, *_ = setup
    ms = [wl.mesh_multiset for wl in test_sc]
    p.perch_set_heuristic_net(net, 8)
    p.perch_search_multi(te, ms, batch_states=2, w=2.0, heuristics=5)
    seconds, states, crops = p.perch_search_stats()
    ev, ab, sel = p.perch_search_times()
    assert states > 0 and crops > 0 and seconds > 0.0
    assert ev > 0.0 and ab > 0.0 and sel > 0.0
    p.perch_search_multi(te, ms, batch_states=2, w=1.0, heuristics=0)
    assert p.perch_search_stats()[1:] == (0, 0)


def test_learned_queue_expands_fewer_states_than_plain_search(setup):
    """What the learned queue adds to the method without it (plain
    uniform-cost search, the paper's exact search): on the held-out scenes
    Focal-MHA* with the anchor and the learned queue (w = 2) never expands
    more states than plain search, expands fewer in all, and returns a scene
    within w times the optimum."""
    p, net, test_sc, te, *_ = setup
    ms = [wl.mesh_multiset for wl in test_sc]
    p.perch_set_heuristic_net(net, 8)
    plain = p.perch_search_multi(te, ms, batch_states=2, w=1.0, heuristics=0)
    learned = p.perch_search_multi(te, ms, batch_states=2, w=2.0, heuristics=4)
    for a, b in zip(plain, learned):
        assert a["proven_optimal"] and b["cost"] <= 2.0 * a["cost"] + 1e-9
        assert b["expansions"] <= a["expansions"]
    assert sum(b["expansions"] for b in learned) < sum(a["expansions"] for a in plain)
