"""Checks of the synthetic workload generator (inputs shared by the oracle
and the CUDA library): closed outward-facing meshes, V(O) inside the solid
(the paper's inscribed-cylinder volume of Sec. III-A must be conservative),
seeded determinism, and the observation statistics of the workloads."""
import numpy as np
import pytest

from paper_1510_05613_gb300 import synth


ALL = synth.meshes_c1() + synth.meshes_c2() + synth.meshes_c3()


@pytest.mark.parametrize("m", ALL, ids=[f"{m.name}{m.n_tris}" for m in ALL])
def test_mesh_closed_and_outward(m):
    t = m.tris.astype(np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    fwd = {tuple(x) for x in e.tolist()}
    assert len(fwd) == len(e)  # no directed edge twice
    assert all((b, a) in fwd for a, b in fwd)  # every edge has its opposite
    v = m.verts.astype(np.float64)
    vol = np.einsum("ij,ij->i", v[t[:, 0]], np.cross(v[t[:, 1]], v[t[:, 2]])).sum() / 6.0
    assert vol > 0


def _inside(m: synth.Mesh, p):
    """Point-in-mesh by ray parity along +x (double precision)."""
    v = m.verts.astype(np.float64)[m.tris]
    a, b, c = v[:, 0], v[:, 1], v[:, 2]
    d = np.array([1.0, 0.3e-3, 0.7e-3])
    e1, e2 = b - a, c - a
    h = np.cross(d, e2)
    det = (e1 * h).sum(1)
    ok = np.abs(det) > 1e-15
    f = np.where(ok, 1.0 / np.where(ok, det, 1), 0)
    s = p - a
    u = f * (s * h).sum(1)
    q = np.cross(s, e1)
    vv = f * (q @ d)
    tt = f * (e2 * q).sum(1)
    hit = ok & (u >= 0) & (u <= 1) & (vv >= 0) & (u + vv <= 1) & (tt > 0)
    return hit.sum() % 2 == 1


@pytest.mark.parametrize("m", ALL, ids=[f"{m.name}{m.n_tris}" for m in ALL])
def test_inscribed_cylinder_inside_mesh(m):
    rng = np.random.default_rng(1)
    th = rng.uniform(0, 2 * np.pi, 60)
    zs = rng.uniform(m.vol_zlo, m.vol_zhi, 60)
    pts = np.stack([m.vol_r * np.cos(th), m.vol_r * np.sin(th), zs], 1)
    # boundary of the cylinder, including its top and bottom rims
    pts = np.concatenate([pts, [[m.vol_r, 0, m.vol_zlo], [0, -m.vol_r, m.vol_zhi]]])
    assert all(_inside(m, p) for p in pts)


def test_splitmix_reference_values():
    # SplitMix64 with seed 0: first outputs (Steele et al. 2014 / Vigna's reference code)
    v = synth.splitmix64(0, 3)
    assert [int(x) for x in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_workloads_are_seeded_and_shaped():
    a, b = synth.workload_c1(), synth.workload_c1()
    assert np.array_equal(a.depth, b.depth) and np.array_equal(a.gt, b.gt)
    assert a.depth.shape == (120, 160)
    frac_missing = 1.0 - (a.depth > 0).sum() / max(1, (synth.raycast_depth(a.cam, a.meshes, a.grid, a.gt) > 0).sum())
    assert 0.0 < frac_missing < 0.15
    assert a.grid.n_poses == 800
    c2 = synth.workload_c2()
    assert c2.depth.shape == (480, 640) and c2.grid.n_poses == 40000
    assert all(9000 <= m.n_tris <= 11000 for m in c2.meshes)


def test_c3_workload_is_heavily_occluded():
    wl = synth.workload_c3()
    assert wl.K == 5 and len(set(int(m) for m in wl.gt["mesh"])) == 5
    occ = np.array(wl.extra["occlusion"])
    assert 0.7 < occ.max() < 1.0
    sizes = sorted(m.n_tris for m in wl.meshes)
    assert sizes[0] <= 2100 and sizes[-1] >= 49000


def test_c2_off_grid_workload():
    wl = synth.workload_c2_off_grid(1)
    j = np.array(wl.extra["jitter"])
    step = float(wl.grid.xs[1] - wl.grid.xs[0])
    assert j.shape == (3, 3)
    assert np.all(np.abs(j[:, :2]) <= 0.5 * step) and np.all(np.abs(j[:, 2]) <= 0.5 * 2 * np.pi / wl.grid.n_yaw)
    assert np.abs(j).max() > 0  # really off the grid
    # footprints stay apart with the offsets (1.5 steps of margin)
    for a in range(3):
        for b in range(a + 1, 3):
            oa, ob = wl.gt[a], wl.gt[b]
            d = np.hypot(float(wl.grid.xs[oa["ix"]] - wl.grid.xs[ob["ix"]]),
                         float(wl.grid.ys[oa["iy"]] - wl.grid.ys[ob["iy"]]))
            assert d > wl.meshes[oa["mesh"]].footprint_radius + wl.meshes[ob["mesh"]].footprint_radius + step
    # the observation is made at the offset poses
    on = synth.raycast_depth(wl.cam, wl.meshes, wl.grid, wl.gt)
    off = synth.raycast_depth(wl.cam, wl.meshes, wl.grid, wl.gt, wl.extra["jitter"])
    assert not np.array_equal(on > 0, off > 0)
    assert np.array_equal(wl.depth, synth.workload_c2_off_grid(1).depth)
