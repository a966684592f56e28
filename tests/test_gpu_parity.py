"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer records (dJr, dJo, residual, violations, |dR|, flags) must be
bit-exact; rendered depths are compared bit for bit as well (the required
tolerance for depths is 1e-4 m, and the arithmetic contract makes them equal).
"""
import numpy as np
import pytest

import oracle
from oracle import search
from paper_1510_05613_gb300 import perch, synth

pytestmark = pytest.mark.gpu


def _recs(out):
    r = perch.records(out)
    r[:, 5] &= 0x7FFFFFFF
    return r


@pytest.fixture(scope="module")
def c1():
    wl = synth.workload_c1()
    p = perch.Perch(0)
    p.setup(wl)
    return wl, p, oracle.World.of(wl)


@pytest.fixture(scope="module")
def c2():
    wl = synth.workload_c2()
    p = perch.Perch(0)
    p.setup(wl)
    return wl, p, oracle.World.of(wl)


def _compare(wl, p, w, parents, hp, hyps, K):
    got = _recs(p.perch_eval_successors(parents, hp, hyps, K))
    exp = oracle.eval_batch(w, wl.depth, parents, hp, hyps, K)
    bad = np.nonzero((got != exp).any(1))[0]
    assert bad.size == 0, f"{bad.size} mismatches, first {hyps[bad[:3]]}: gpu {got[bad[:3]]} oracle {exp[bad[:3]]}"
    return got


def test_render_bit_exact_c1(c1):
    wl, p, w = c1
    for objs in (wl.gt, wl.gt[:1], wl.gt[::-1]):
        z, culled = p.perch_render(objs)
        ze, ce = oracle.render(w, objs)
        assert culled == ce
        assert np.array_equal(z.view(np.uint32), ze.view(np.uint32))


def test_render_bit_exact_c2(c2):
    wl, p, w = c2
    z, culled = p.perch_render(wl.gt)
    ze, ce = oracle.render(w, wl.gt)
    assert culled == ce
    assert np.array_equal(z.view(np.uint32), ze.view(np.uint32))
    fin = np.isfinite(ze)
    assert np.max(np.abs(z[fin] - ze[fin])) <= 1e-4


def test_c1_level0_all_hypotheses(c1):
    wl, p, w = c1
    hyps = synth.all_hypotheses(wl.grid, [0, 1])
    got = _compare(wl, p, w, [wl.gt[:0]], np.zeros(len(hyps), np.int32), hyps, wl.K)
    assert (got[:, 0] > 0).any() and (got[:, 1] > 0).any()


def test_c1_last_level_with_residual(c1):
    wl, p, w = c1
    parents = [wl.gt[:1], wl.gt[1:2]]
    h0 = synth.all_hypotheses(wl.grid, [int(wl.gt[1]["mesh"])])
    h1 = synth.all_hypotheses(wl.grid, [int(wl.gt[0]["mesh"])])
    hyps = np.concatenate([h0, h1])
    hp = np.concatenate([np.zeros(len(h0), np.int32), np.ones(len(h1), np.int32)])
    got = _compare(wl, p, w, parents, hp, hyps, wl.K)
    assert (got[:, 2] > 0).any() and (got[:, 3] > 0).any()


def test_c1_mixed_parents_and_levels(c1):
    wl, p, w = c1
    rng = np.random.default_rng(0)
    allh = synth.all_hypotheses(wl.grid, [0, 1])
    parents = [wl.gt[:0], wl.gt[:1], allh[rng.choice(len(allh), 1)], allh[rng.choice(len(allh), 1)]]
    n = 700
    hyps = allh[rng.choice(len(allh), n)]
    hp = rng.integers(0, len(parents), n).astype(np.int32)
    _compare(wl, p, w, parents, hp, hyps, 2)
    # the same batch with K = 3 (no residual anywhere) and K = 1 from the root
    _compare(wl, p, w, parents, hp, hyps, 3)
    _compare(wl, p, w, [wl.gt[:0]], np.zeros(200, np.int32), hyps[:200], 1)


def test_c2_sampled_all_levels(c2):
    wl, p, w = c2
    rng = np.random.default_rng(1)
    allh = synth.all_hypotheses(wl.grid, [0, 1, 2])
    # near the ground truth (overlapping the observation) and uniform
    near = []
    for o in wl.gt:
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for k in (0, 3, 8):
                    near.append((int(o["mesh"]), int(o["ix"]) + dx, int(o["iy"]) + dy, (int(o["iyaw"]) + k) % 16))
    hyps = np.concatenate([synth.objs(near), allh[rng.choice(len(allh), 120)]])
    parents = [wl.gt[:0], wl.gt[:1], wl.gt[:2]]
    hp = np.repeat(np.arange(3, dtype=np.int32), len(hyps))
    got = _compare(wl, p, w, parents, hp, np.tile(hyps, 3), 3)
    assert (got[:, 1] > 0).any() and (got[:, 2] > 0).any()


def test_c2_bench_launch_sampled(c2):
    """The full-size batch the benchmark times (root 120k + level-1 80k +
    level-2 40k hypotheses, one launch): sampled records against the oracle,
    invariants on all of them."""
    wl, p, w = c2
    from bench import c2_batch
    parents, hp, hyps = c2_batch(wl)
    got = _recs(p.perch_eval_successors(parents, hp, hyps, wl.K))
    assert got.shape == (len(hyps), 7)
    # invariants on every record
    inval = got[:, 3] > 0
    assert np.all((got[:, 5] & 2 > 0) == inval)
    assert np.all(got[inval, :3] == 0)
    assert np.all(got[~inval, 0] <= got[~inval, 4])
    assert np.all(got[hp == 0, 3] == 0) and np.all(got[hp != 2, 2] == 0)
    # sampled exact parity
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(len(hyps), 150, replace=False))
    exp = oracle.eval_batch(w, wl.depth, parents, hp[idx], hyps[idx], wl.K)
    assert np.array_equal(got[idx], exp)


def test_shared_renders_identical_to_per_hypothesis_renders(c2):
    """A successor's new-object render depends on its mesh and pose alone
    (Sec. III-A, R_j), so rendering each distinct pose of a batch once and
    costing every hypothesis from that tile must give the records of
    rendering every hypothesis: checked on a batch whose poses repeat over
    four parents (root, middle level, last level), with the exact shortcut
    off and on, and against the oracle on a sample."""
    wl, p, w = c2
    rng = np.random.default_rng(21)
    parents = [wl.gt[:0], wl.gt[:1], wl.gt[:2], wl.gt[1:2]]
    allh = synth.all_hypotheses(wl.grid, [0, 1, 2])
    poses = allh[rng.choice(len(allh), 2500, replace=False)]
    near = np.concatenate([wl.gt, allh[np.isin(allh["ix"], wl.gt["ix"]) & np.isin(allh["iy"], wl.gt["iy"])][:500]])
    poses = np.concatenate([poses, near])
    reps = rng.integers(1, 5, len(poses))  # 1-4 parents per pose
    hyps = np.repeat(poses, reps)
    hp = np.concatenate([rng.choice(4, r, replace=False) for r in reps]).astype(np.int32)
    try:
        for short in (False, True):
            p.perch_set_shortcut(short)
            p.perch_set_share_renders(True)
            a = _recs(p.perch_eval_successors(parents, hp, hyps, wl.K))
            assert p.perch_last_phase_times()[1]
            p.perch_set_share_renders(False)
            b = _recs(p.perch_eval_successors(parents, hp, hyps, wl.K))
            assert not p.perch_last_phase_times()[1]
            assert np.array_equal(a, b)
    finally:
        p.perch_set_shortcut(True)
        p.perch_set_share_renders(True)
    pick = rng.choice(len(hyps), 150, replace=False)
    exp = oracle.eval_batch(w, wl.depth, parents, hp[pick], hyps[pick], wl.K)
    assert np.array_equal(a[pick], exp)
    assert (a[:, 3] > 0).any() and (a[:, 2] > 0).any() and (a[:, 1] > 0).any()


def test_render_cache_keeps_records(c2):
    """With the render cache on, each pose's stored render is kept across
    evaluations; a render depends on its mesh and pose (and its explained
    flags on the observation), so batches that repeat and mix poses over
    other parents, a single-parent batch and the first batch again give the
    records of evaluating without it. A new observation empties the cache
    (the explained flags change), checked against a cache-off evaluation of
    that observation, and against the oracle on a sample."""
    wl, p, w = c2
    rng = np.random.default_rng(41)
    wl2 = synth.workload_c2(scene=1)
    allh = synth.all_hypotheses(wl.grid, [0, 1, 2])
    near = np.concatenate([_near(wl.grid, wl.gt, {0, 1, 2}), _near(wl.grid, wl2.gt, {0, 1, 2})])
    A = np.concatenate([allh[rng.choice(len(allh), 3000, replace=False)], near])
    B = np.concatenate([A[::2], allh[rng.choice(len(allh), 1500, replace=False)]])
    batches = [([wl.gt[:0], wl.gt[:1]], A), ([wl.gt[:2], wl.gt[:0], wl.gt[1:2]], B), ([wl.gt[:1]], B),
               ([wl.gt[:0], wl.gt[:1]], A)]
    hps = [rng.integers(0, len(par), len(h)).astype(np.int32) for par, h in batches]

    def run():
        return [_recs(p.perch_eval_successors(par, hp, h, wl.K)) for (par, h), hp in zip(batches, hps)]

    try:
        p.perch_set_shortcut(False)
        ref = run()
        p.perch_set_render_cache(True)
        got = run()
        for k, (a, b) in enumerate(zip(ref, got)):
            assert np.array_equal(a, b), k
        p.perch_eval_successors(batches[2][0], hps[2], batches[2][1], wl.K)
        assert p.perch_last_phase_times()[1]  # one parent, yet shared renders (from the cache)
        p.perch_set_observation(wl2.depth, wl2.cam.fxfycxcy, wl2.cam.T_wc, wl2.delta)
        got2 = run()
        p.perch_set_render_cache(False)
        ref2 = run()
        for k, (a, b) in enumerate(zip(ref2, got2)):
            assert np.array_equal(a, b), k
        assert any(not np.array_equal(a, b) for a, b in zip(ref, ref2))  # the observation matters
    finally:
        p.perch_set_render_cache(False)
        p.perch_set_shortcut(True)
        p.perch_set_observation(wl.depth, wl.cam.fxfycxcy, wl.cam.T_wc, wl.delta)
    pick = rng.choice(len(A), 100, replace=False)
    exp = oracle.eval_batch(w, wl.depth, batches[3][0], hps[3][pick], A[pick], wl.K)
    assert np.array_equal(got[3][pick], exp)


def test_render_cache_search_unchanged(c1):
    """Uniform-cost search with the render cache on returns the same scene,
    cost, expansions and successors as without it; with one state per batch
    (single-parent batches, which the cache sends through shared renders)
    the same scene and cost."""
    wl, p, w = c1
    base = p.perch_search(wl.mesh_multiset, batch_states=4)
    p.perch_set_render_cache(True)
    try:
        r = p.perch_search(wl.mesh_multiset, batch_states=4)
        r1 = p.perch_search(wl.mesh_multiset, batch_states=1)
    finally:
        p.perch_set_render_cache(False)
    for k in ("cost", "key", "expansions", "successors", "proven_optimal"):
        assert r[k] == base[k], k
    assert (r1["cost"], r1["key"]) == (base["cost"], base["key"]) and r1["proven_optimal"]


def _near(grid, objs, types):
    """Hypotheses at and around the ground-truth poses of the given types
    (one grid step and one yaw step away), where V(O) holds observed points."""
    out = []
    for o in objs:
        if int(o["mesh"]) not in types:
            continue
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dk in (-1, 0, 1):
                    ix, iy = int(o["ix"]) + dx, int(o["iy"]) + dy
                    if 0 <= ix < grid.nx and 0 <= iy < grid.ny:
                        out.append((int(o["mesh"]), ix, iy, (int(o["iyaw"]) + dk) % grid.n_yaw))
    return synth.objs(out)


@pytest.mark.parametrize("which", ["c1", "c2", "c3"])
def test_closed_form_volumes_bit_exact(which):
    """V(O) in closed form (box, regular prism, superquadric; Sec. III-A):
    records bit-exact with the oracle's closed forms at the root, a middle
    level and the last level (residual), on random poses and on poses around
    the ground truth; the closed forms change n_vol and dJ_o there; switching
    back restores the inscribed cylinders' records."""
    wl = {"c1": synth.workload_c1, "c2": synth.workload_c2, "c3": synth.workload_c3}[which]()
    p = perch.Perch(0)
    p.setup(wl, exact_volumes=True)
    we, wc = oracle.World.of(wl, exact_volumes=True), oracle.World.of(wl)
    rng = np.random.default_rng(8)
    K = wl.K
    parents = [wl.gt[:0], wl.gt[:1], wl.gt[:K - 1]]
    hyps, hp = [], []
    for i, par in enumerate(parents):
        rem = list(wl.mesh_multiset)
        for m in par["mesh"]:
            rem.remove(int(m))
        types = sorted(set(rem))
        allh = synth.all_hypotheses(wl.grid, types)
        n = len(allh) if which == "c1" else 120
        pick = allh[rng.choice(len(allh), n, replace=False)]
        near = _near(wl.grid, wl.gt, set(types))
        hyps += [pick, near]
        hp += [np.full(len(pick) + len(near), i, np.int32)]
    hyps, hp = np.concatenate(hyps), np.concatenate(hp)
    try:
        got = _recs(p.perch_eval_successors(parents, hp, hyps, K))
        exp = oracle.eval_batch(we, wl.depth, parents, hp, hyps, K)
        bad = np.nonzero((got != exp).any(1))[0]
        assert bad.size == 0, f"{bad.size} mismatches, first {hyps[bad[:3]]}: gpu {got[bad[:3]]} oracle {exp[bad[:3]]}"
        cyl = oracle.eval_batch(wc, wl.depth, parents, hp, hyps, K)
        assert (exp[:, 6] != cyl[:, 6]).sum() > 10 and (exp[:, 1] != cyl[:, 1]).any()
        p.perch_set_volumes(None)
        back = _recs(p.perch_eval_successors(parents, hp, hyps, K))
        assert np.array_equal(back, cyl)
    finally:
        p.close()


def test_shortcut_records_identical_and_taken(c2):
    """The exact shortcut (hypotheses far from the observation and from the
    parent's render) gives the same records as rendering every hypothesis,
    on the full benchmark batch, and takes most of it."""
    wl, p, w = c2
    from bench import c2_batch
    parents, hp, hyps = c2_batch(wl)
    p.perch_set_shortcut(False)
    full = _recs(p.perch_eval_successors(parents, hp, hyps, wl.K))
    assert p.perch_shortcut_stats() == (0, len(hyps))
    p.perch_set_shortcut(True)
    fast = _recs(p.perch_eval_successors(parents, hp, hyps, wl.K))
    n_short, n = p.perch_shortcut_stats()
    assert n == len(hyps) and n_short > len(hyps) // 2
    bad = np.nonzero((full != fast).any(1))[0]
    assert bad.size == 0, (bad[:5], full[bad[:3]], fast[bad[:3]])


def test_shortcut_multi_scene_identical():
    meshes = synth.meshes_c3()[:4]
    grid = synth.pose_grid(-0.49, 0.04, 25, 8)
    wls = synth.workloads_c5(3, grid=grid, meshes=meshes, k_range=(2, 3))
    p = perch.Perch(0)
    p.setup(wls[0])
    for s, wl in enumerate(wls[1:], 1):
        p.perch_set_scene(s, wl.depth)
    parents, ps, pk, hp, hyps = [], [], [], [], []
    rng = np.random.default_rng(7)
    for s, wl in enumerate(wls):
        for j in range(wl.K):
            h = synth.all_hypotheses(grid, sorted(set(int(m) for m in wl.gt["mesh"][j:])))
            h = h[rng.choice(len(h), min(len(h), 3000), replace=False)]
            hp.append(np.full(len(h), len(parents), np.int32))
            hyps.append(h)
            parents.append(wl.gt[:j])
            ps.append(s)
            pk.append(wl.K)
    hp, hyps = np.concatenate(hp), np.concatenate(hyps)
    p.perch_set_shortcut(False)
    full = _recs(p.perch_eval_successors_multi(parents, ps, pk, hp, hyps))
    p.perch_set_shortcut(True)
    fast = _recs(p.perch_eval_successors_multi(parents, ps, pk, hp, hyps))
    assert p.perch_shortcut_stats()[0] > len(hyps) // 3
    assert np.array_equal(full, fast)
    # sampled records of every parent against the oracle (shortcut on)
    for s, wl in enumerate(wls):
        wo = oracle.World.of(wl)
        for j in range(wl.K):
            pi = [i for i in range(len(parents)) if ps[i] == s and len(parents[i]) == j][0]
            idx = np.nonzero(hp == pi)[0][::97]
            exp = oracle.eval_batch(wo, wl.depth, [parents[pi]], np.zeros(len(idx), np.int32), hyps[idx], wl.K)
            assert np.array_equal(fast[idx], exp)


def test_empty_observation_and_huge_delta():
    wl = synth.workload_c1()
    allh = synth.all_hypotheses(wl.grid, [0, 1])[::7]
    for depth, delta in ((np.zeros_like(wl.depth), 0.01), (wl.depth, 5.0)):
        p = perch.Perch(0)
        p.perch_load_meshes(wl.meshes)
        p.perch_set_pose_grid(wl.grid)
        p.perch_set_observation(depth, wl.cam.fxfycxcy, wl.cam.T_wc, delta)
        w = oracle.World(wl.cam, wl.meshes, wl.grid, delta)
        parents = [wl.gt[:0], wl.gt[:1]]
        hp = np.arange(len(allh), dtype=np.int32) % 2
        got = _recs(p.perch_eval_successors(parents, hp, allh, 2))
        exp = oracle.eval_batch(w, depth, parents, hp, allh, 2)
        assert np.array_equal(got, exp)
        p.close()


def test_offscreen_and_ragged_pose_grid():
    """A pose grid reaching past the image edge (partly and fully off-screen
    objects) and an odd number of poses."""
    wl = synth.workload_c1()
    grid = synth.pose_grid(-0.9, 0.13, 13, 5)
    p = perch.Perch(0)
    p.perch_load_meshes(wl.meshes)
    p.perch_set_pose_grid(grid)
    p.perch_set_observation(wl.depth, wl.cam.fxfycxcy, wl.cam.T_wc, wl.delta)
    w = oracle.World(wl.cam, wl.meshes, grid, wl.delta)
    hyps = synth.all_hypotheses(grid, [0, 1])
    parent = synth.objs([(0, 6, 6, 0)])
    hp = np.arange(len(hyps), dtype=np.int32) % 2
    got = _recs(p.perch_eval_successors([parent[:0], parent], hp, hyps, 2))
    exp = oracle.eval_batch(w, wl.depth, [parent[:0], parent], hp, hyps, 2)
    assert np.array_equal(got, exp)
    assert (got[:, 4] == 0).any()  # some hypotheses fully off-screen
    p.close()


def test_device_pointer_entry_point(c1):
    import torch
    wl, p, w = c1
    hyps = synth.all_hypotheses(wl.grid, [0, 1])[::3]
    P, plen, stride = perch.Perch.pack_parents([wl.gt[:1]])
    dev = torch.device("cuda:0")
    tP = torch.from_numpy(P.view(np.int16).reshape(-1).copy()).to(dev)
    tplen = torch.from_numpy(plen).to(dev)
    thp = torch.zeros(len(hyps), dtype=torch.int32, device=dev)
    th = torch.from_numpy(np.ascontiguousarray(hyps).view(np.int16).reshape(-1).copy()).to(dev)
    tout = torch.zeros(len(hyps) * 7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    p.perch_eval_successors_dev(tP, stride, tplen, thp, th, 2, tout)
    torch.cuda.synchronize()
    got = tout.cpu().numpy().reshape(-1, 7).astype(np.int64)
    exp = oracle.eval_batch(w, wl.depth, [wl.gt[:1]], np.zeros(len(hyps), np.int32), hyps, 2)
    assert np.array_equal(got, exp)


def test_argument_errors(c1):
    wl, p, w = c1
    hyps = synth.all_hypotheses(wl.grid, [0])[:4]
    with pytest.raises(perch.PerchError) as e:
        p.perch_eval_successors([wl.gt[:0]], np.array([0, 0, 0, 5], np.int32), hyps, 2)
    assert e.value.code == perch.PERCH_E_ARG
    bad = hyps.copy()
    bad["ix"][1] = 99
    with pytest.raises(perch.PerchError):
        p.perch_eval_successors([wl.gt[:0]], np.zeros(4, np.int32), bad, 2)
    with pytest.raises(perch.PerchError):  # parent as long as the full scene
        p.perch_eval_successors([wl.gt], np.zeros(4, np.int32), hyps, 2)
    assert len(p.perch_eval_successors([wl.gt[:0]], np.zeros(0, np.int32), hyps[:0], 2)) == 0
    with pytest.raises(perch.PerchError) as e:  # no heuristic bit 5
        p.perch_search(wl.mesh_multiset, heuristics=32)
    assert e.value.code == perch.PERCH_E_ARG


def test_wait_limit_failure_path_reports_and_recovers(c1):
    """A bounded wait of the evaluation kernel that gives up (limit 0 polls:
    every first wait for a bulk copy gives up at once) leaves records with
    flags bit 30 and no cost; the host call and the search return
    PERCH_E_DEVICE instead of a result. The kernel drains every copy in
    flight before it goes on, so the context stays usable: with the default
    limit the records equal the oracle's again."""
    import torch
    wl, p, w = c1
    hyps = synth.all_hypotheses(wl.grid, [0, 1])[::5]
    hp = np.zeros(len(hyps), np.int32)
    dev = torch.device("cuda:0")
    P, plen, stride = perch.Perch.pack_parents([wl.gt[:1]])
    tP = torch.from_numpy(P.view(np.int16).reshape(-1).copy()).to(dev)
    tplen = torch.from_numpy(plen).to(dev)
    thp = torch.zeros(len(hyps), dtype=torch.int32, device=dev)
    th = torch.from_numpy(np.ascontiguousarray(hyps).view(np.int16).reshape(-1).copy()).to(dev)
    tout = torch.full((len(hyps) * 7,), -7, dtype=torch.int32, device=dev)
    p.perch_set_shortcut(False)
    try:
        p.perch_set_wait_limit(0)
        with pytest.raises(perch.PerchError) as e:
            p.perch_eval_successors([wl.gt[:0]], hp, hyps, wl.K)
        assert e.value.code == perch.PERCH_E_DEVICE
        torch.cuda.synchronize()
        p.perch_eval_successors_dev(tP, stride, tplen, thp, th, wl.K, tout)
        torch.cuda.synchronize()
        got = tout.cpu().numpy().reshape(-1, 7)
        assert (got[:, 5].astype(np.uint32) == perch.FLAG_TIMEOUT).all()  # every record: bit 30 and nothing else
        assert (got[:, [0, 1, 2, 3, 4, 6]] == 0).all()
        with pytest.raises(perch.PerchError) as e:
            p.perch_search(wl.mesh_multiset, batch_states=4)
        assert e.value.code == perch.PERCH_E_DEVICE
    finally:
        p.perch_set_wait_limit(-1)
        p.perch_set_shortcut(True)
    _compare(wl, p, w, [wl.gt[:0]], hp, hyps, wl.K)
    p.perch_eval_successors_dev(tP, stride, tplen, thp, th, wl.K, tout)
    torch.cuda.synchronize()
    exp = oracle.eval_batch(w, wl.depth, [wl.gt[:1]], hp, hyps, wl.K)
    assert np.array_equal(tout.cpu().numpy().reshape(-1, 7).astype(np.int64), exp)


def test_search_matches_oracle_exhaustive_small_c1():
    grid = synth.pose_grid(-0.15, 0.1, 4, 4)
    wl = synth.workload_c1(scene=3, grid=grid)
    p = perch.Perch(0)
    p.setup(wl)
    w = oracle.World.of(wl)
    ex_cost, ex_key = search.exhaustive(w, wl.depth, wl.grid, wl.mesh_multiset)
    for B in (1, 3, 64):
        for heur in (0, 16):  # 16: a greedy incumbent first; the same optimum
            r = p.perch_search(wl.mesh_multiset, batch_states=B, heuristics=heur)
            assert r["proven_optimal"] and (r["cost"], r["key"]) == (ex_cost, ex_key), (B, heur)
    p.close()


def test_search_matches_oracle_ucs_full_c1(c1):
    wl, p, w = c1
    cost, key, _ = search.uniform_cost_search(w, wl.depth, wl.grid, wl.mesh_multiset)
    r = p.perch_search(wl.mesh_multiset, batch_states=16)
    assert r["proven_optimal"] and (r["cost"], r["key"]) == (cost, key)
    # with the greedy incumbent first: the same optimum, and no more successors kept
    ri = p.perch_search(wl.mesh_multiset, batch_states=16, heuristics=16)
    assert ri["proven_optimal"] and (ri["cost"], ri["key"]) == (cost, key)


def test_render_launch_parameters_do_not_change_records():
    """The render's CTA width, inline limit (which triangles a lane
    rasterises itself and which a warp takes from the queue) and bin depth
    (how many the queue holds before a lane rasterises one) change only who
    writes a pixel's depth, never the depth; the cost kernel's stage buffers
    (one, or two so that the next tile is copied while the current one is
    costed) change only when a tile arrives. The same records for every
    setting the autotuner can pick, on the uneven meshes of the
    heavy-occlusion workload (2k-50k triangles), checked against the oracle
    on a sample."""
    wl = synth.workload_c3()
    p = perch.Perch(0)
    p.setup(wl)
    w = oracle.World.of(wl)
    rng = np.random.default_rng(31)
    parents = [wl.gt[:0], wl.gt[:2]]
    hyps, hp = [], []
    for i, par in enumerate(parents):
        rem = list(wl.mesh_multiset)
        for m in par["mesh"]:
            rem.remove(int(m))
        allh = synth.all_hypotheses(wl.grid, sorted(set(rem)))
        pick = allh[rng.choice(len(allh), 1500, replace=False)]
        near = _near(wl.grid, wl.gt, set(rem))
        hyps += [pick, near]
        hp += [np.full(len(pick) + len(near), i, np.int32)]
    hyps, hp = np.concatenate(hyps), np.concatenate(hp)
    ref = None
    try:
        p.perch_set_shortcut(False)
        for threads, inl, bins, stages in ((256, 16, 128, 1), (128, 8, 32, 2), (512, 32, 64, 1), (256, 32, 32, 2),
                                           (128, 16, 64, 2)):
            p.perch_set_threads(threads)
            p.perch_set_inline_pixels(inl)
            p.perch_set_bin_depth(bins)
            p.perch_set_cost_stages(stages)
            assert p.perch_launch_config()[:2] == ([threads] * len(wl.meshes), [inl] * len(wl.meshes))
            assert p.perch_launch_bin_depths() == [bins] * len(wl.meshes)
            got = _recs(p.perch_eval_successors(parents, hp, hyps, wl.K))
            if ref is None:
                ref = got
            assert np.array_equal(got, ref), (threads, inl, bins, stages)
    finally:
        p.close()
    pick = rng.choice(len(hyps), 60, replace=False)
    assert np.array_equal(ref[pick], oracle.eval_batch(w, wl.depth, parents, hp[pick], hyps[pick], wl.K))


def test_symmetric_search_matches_oracle_c1(c1):
    """With the meshes' rotational symmetry declared, the GPU search places a
    symmetric mesh only at the yaws no smaller yaw equals modulo its symmetry
    (Sec. IV-E) and returns the oracle's optimum of that tree, evaluating
    fewer successors than the full tree."""
    wl, p, w = c1
    yaws = search.symmetric_yaws(wl.grid, [m.sym for m in wl.meshes])
    cost, key, _ = search.uniform_cost_search(w, wl.depth, wl.grid, wl.mesh_multiset, yaws=yaws)
    full = p.perch_search(wl.mesh_multiset, batch_states=16)
    p.perch_set_symmetry(wl.meshes)
    try:
        r = p.perch_search(wl.mesh_multiset, batch_states=16)
    finally:
        p.perch_set_symmetry(None)
    assert r["proven_optimal"] and (r["cost"], r["key"]) == (cost, key)
    assert all(o[3] in yaws[o[0]] for o in r["key"])
    assert r["successors"] < 0.6 * full["successors"]


def test_c3_uneven_meshes_sampled():
    """Heavy-occlusion workload: five of eight meshes of 2k-50k triangles;
    sampled records at the root, a middle level and the last level."""
    wl = synth.workload_c3()
    p = perch.Perch(0)
    p.setup(wl)
    w = oracle.World.of(wl)
    rng = np.random.default_rng(3)
    parents = [wl.gt[:0], wl.gt[:2], wl.gt[:4]]
    hyps, hp = [], []
    for i, par in enumerate(parents):
        rem = sorted(set(int(m) for m in wl.gt["mesh"]) - set(int(m) for m in par["mesh"]))
        allh = synth.all_hypotheses(wl.grid, rem)
        pick = allh[rng.choice(len(allh), 40, replace=False)]
        near = [o for o in wl.gt if int(o["mesh"]) in rem]
        hyps += [pick, np.array(near, synth.OBJ_DTYPE)]
        hp += [np.full(len(pick) + len(near), i, np.int32)]
    hyps, hp = np.concatenate(hyps), np.concatenate(hp)
    got = _compare(wl, p, w, parents, hp, hyps, wl.K)
    assert (got[:, 2] > 0).any()
    p.close()


def _dev_batch(torch, parents, hp, hyps):
    dev = torch.device("cuda:0")
    P, plen, stride = perch.Perch.pack_parents(parents)
    tP = torch.from_numpy(P.view(np.int16).reshape(-1).copy()).to(dev)
    th = torch.from_numpy(np.ascontiguousarray(hyps).view(np.int16).reshape(-1).copy()).to(dev)
    return tP, stride, torch.from_numpy(plen).to(dev), torch.from_numpy(np.ascontiguousarray(hp)).to(dev), th


def test_graph_and_autotune_match_oracle(c2):
    """The CUDA-graph entry point and autotuned launch widths give the same
    records as the oracle; replaying the graph after rewriting the
    hypotheses in place evaluates the new ones."""
    import torch
    wl, _, w = c2
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    p = perch.Perch(0, stream=stream.cuda_stream)
    p.setup(wl)
    widths = p.perch_autotune(256)
    assert len(widths) == 3 and set(widths) <= {128, 256, 512}
    rng = np.random.default_rng(9)
    allh = synth.all_hypotheses(wl.grid, [0, 1, 2])
    parents = [wl.gt[:0], wl.gt[:2]]
    hp = rng.integers(0, 2, 90).astype(np.int32)
    outs = []
    for rep in range(2):
        hyps = allh[rng.choice(len(allh), 90, replace=False)]
        hyps["mesh"] = np.where(hp == 1, 2, hyps["mesh"])  # the 2-object parent needs the third type
        tP, stride, tplen, thp, th = _dev_batch(torch, parents, hp, hyps)
        if rep == 0:
            keep = (tP, tplen, thp, th)
            tout = torch.zeros(len(hyps) * 7, dtype=torch.int32, device="cuda:0")
        else:
            keep[3].copy_(th)  # same device buffers, new contents
        p.perch_eval_graph(keep[0], stride, keep[1], keep[2], keep[3], wl.K, tout)
        torch.cuda.synchronize()
        got = tout.cpu().numpy().reshape(-1, 7).astype(np.int64)
        exp = oracle.eval_batch(w, wl.depth, parents, hp, hyps, wl.K)
        assert np.array_equal(got, exp)
        outs.append(got)
    assert not np.array_equal(outs[0], outs[1])
    p.close()


def _multi_c1(n):
    """n small independent scenes sharing the C1 camera and meshes."""
    cam, meshes = synth.camera_c1(), synth.meshes_c1()
    grid = synth.pose_grid(-0.15, 0.1, 4, 4)
    return synth.workloads_c5(n, grid=grid, cam=cam, meshes=meshes, k_range=(1, 2))


def test_multi_scene_eval_matches_oracle():
    wls = _multi_c1(5)
    p = perch.Perch(0)
    p.setup(wls[0])
    for s, wl in enumerate(wls[1:], 1):
        p.perch_set_scene(s, wl.depth)
    rng = np.random.default_rng(4)
    allh = synth.all_hypotheses(wls[0].grid, [0, 1])
    parents, pscene, pK = [], [], []
    for s, wl in enumerate(wls):
        parents += [wl.gt[:0], wl.gt[:1]]
        pscene += [s, s]
        pK += [max(wl.K, 2), max(wl.K, 2)]
    hp = rng.integers(0, len(parents), 400).astype(np.int32)
    hyps = allh[rng.choice(len(allh), 400)]
    got = _recs(p.perch_eval_successors_multi(parents, pscene, pK, hp, hyps))
    p.perch_set_render_cache(True)  # plain z kept across the two calls; the same records
    for _ in range(2):
        assert np.array_equal(_recs(p.perch_eval_successors_multi(parents, pscene, pK, hp, hyps)), got)
    p.perch_set_render_cache(False)
    for s, wl in enumerate(wls):
        w = oracle.World.of(wl)
        for j in (2 * s, 2 * s + 1):
            sel = hp == j
            exp = oracle.eval_batch(w, wl.depth, [parents[j]], np.zeros(sel.sum(), np.int32), hyps[sel], pK[j])
            assert np.array_equal(got[sel], exp), (s, j)
    p.close()


def test_multi_scene_search_matches_oracle():
    wls = _multi_c1(6)
    p = perch.Perch(0)
    p.setup(wls[0])
    for s, wl in enumerate(wls[1:], 1):
        p.perch_set_scene(s, wl.depth)
    res = p.perch_search_multi(list(range(len(wls))), [wl.mesh_multiset for wl in wls], batch_states=2,
                               max_hyps_per_launch=300)
    inc = p.perch_search_multi(list(range(len(wls))), [wl.mesh_multiset for wl in wls], batch_states=2,
                               max_hyps_per_launch=300, heuristics=16)
    for wl, r, ri in zip(wls, res, inc):
        w = oracle.World.of(wl)
        cost, key = search.exhaustive(w, wl.depth, wl.grid, wl.mesh_multiset)
        assert r["proven_optimal"] and (r["cost"], r["key"]) == (cost, key)
        assert ri["proven_optimal"] and (ri["cost"], ri["key"]) == (cost, key)
    p.close()


@pytest.mark.parametrize("w,heur", [(1.0, 3), (1.5, 3), (3.0, 3), (3.0, 1), (3.0, 2), (3.0, 19), (1.0, 16)])
def test_focal_mha_search_bound(w, heur):
    """Library Focal-MHA* on the reduced 2-object grid: cost within w times
    the exhaustive optimum (Theorem 2); with w = 1 exactly optimal."""
    grid = synth.pose_grid(-0.15, 0.1, 4, 4)
    wl = synth.workload_c1(scene=3, grid=grid)
    p = perch.Perch(0)
    p.setup(wl)
    wo = oracle.World.of(wl)
    opt, opt_key = search.exhaustive(wo, wl.depth, wl.grid, wl.mesh_multiset)
    r = p.perch_search(wl.mesh_multiset, w=w, heuristics=heur, batch_states=2)
    assert r["status"] == perch.PERCH_OK and opt <= r["cost"] <= w * opt
    if w == 1.0:
        assert (r["cost"], r["key"]) == (opt, opt_key) and r["proven_optimal"]
    p.close()


def test_focal_mha_full_c1_fewer_expansions(c1):
    """On the full 800-pose C1 tree, w = 3 with both heuristics stays within
    the bound and expands no more states than the exact search."""
    wl, p, w = c1
    cost, key, _ = search.uniform_cost_search(w, wl.depth, wl.grid, wl.mesh_multiset)
    exact = p.perch_search(wl.mesh_multiset, batch_states=4)
    fast = p.perch_search(wl.mesh_multiset, w=3.0, heuristics=3, batch_states=4)
    assert exact["cost"] == cost and cost <= fast["cost"] <= 3 * cost
    assert fast["expansions"] <= exact["expansions"]


@pytest.mark.parametrize("heur,w", [(0, 1.0), (3, 3.0)])
def test_multi_scene_search_threads_do_not_change_results(heur, w):
    """Scenes searched together (batches of >= 64k hypotheses, built and
    absorbed by host threads, one scene per thread) give exactly the results
    of each scene searched alone (small batches, one thread): the same cost,
    scene, expansions and successors. Without a launch cap every scene
    expands the same states per round either way."""
    grid = synth.pose_grid(-0.48, 0.04, 25, 8)
    wls = synth.workloads_c5(6, grid=grid, k_range=(3, 3))
    p = perch.Perch(0)
    p.setup(wls[0])
    for s, wl in enumerate(wls[1:], 1):
        p.perch_set_scene(s, wl.depth)
    ids, ms = list(range(len(wls))), [wl.mesh_multiset for wl in wls]
    joint = p.perch_search_multi(ids, ms, batch_states=2, w=w, heuristics=heur)
    assert len(wls) * 3 * grid.n_poses >= 65536  # the root batch alone engages the threads
    for sid, m, r in zip(ids, ms, joint):
        solo = p.perch_search_multi([sid], [m], batch_states=2, w=w, heuristics=heur)[0]
        for k in ("cost", "key", "expansions", "successors", "proven_optimal"):
            assert solo[k] == r[k], (sid, k, solo[k], r[k])
