"""The allocation-free evaluation entry point, through the C ABI.

perch_eval_successors_noalloc is for callers that cannot allocate device
memory when they evaluate successors (a real-time loop that must not stall on
cudaMalloc, or a process whose GPU memory is fixed after start-up); its
scratch is a fixed array inside the library. The call must leave the
device's free memory unchanged, and its records must equal those of
perch_eval_successors_dev on the same inputs, bit for bit (the tolerance of
every record test here), on two calls in a row: the second call must not see
the first call's z-buffers or residual sets, which stay in the shared array.
This file is named to run last.
"""
import numpy as np
import pytest

from paper_1510_05613_gb300 import perch, synth

pytestmark = pytest.mark.gpu


def _dev(torch, a, dev):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.uint8).reshape(-1).copy()).to(dev)


def test_noalloc_matches_existing_entry_point_twice():
    import torch
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    wl = synth.workload_c1()
    p = perch.Perch(0, stream=stream.cuda_stream)
    p.setup(wl)
    allh = synth.all_hypotheses(wl.grid, [0, 1])
    rng = np.random.default_rng(5)
    calls = [
        ([wl.gt[:0], wl.gt[:1], wl.gt[1:2]], rng.choice(len(allh), 1200)),  # root + two last-level parents
        ([wl.gt[1:2], wl.gt[:0]], rng.choice(len(allh), 700)),  # different parents and order
    ]
    for parents, pick in calls:
        hyps = allh[pick]
        hp = rng.integers(0, len(parents), len(hyps)).astype(np.int32)
        P, plen, stride = perch.Perch.pack_parents(parents)
        tP, tplen = _dev(torch, P, dev), torch.from_numpy(plen).to(dev)
        thp, th = torch.from_numpy(hp).to(dev), _dev(torch, hyps, dev)
        ref = torch.full((len(hyps) * 7,), -7, dtype=torch.int32, device=dev)
        got = torch.full((len(hyps) * 7,), -7, dtype=torch.int32, device=dev)
        p.perch_eval_successors_dev(tP, stride, tplen, thp, th, wl.K, ref)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(dev)[0]
        p.perch_eval_successors_noalloc(tP, stride, tplen, thp, th, wl.K, got)
        torch.cuda.synchronize()
        # the call allocated nothing on the device (its set-up was done by
        # perch_set_observation inside p.setup)
        assert torch.cuda.mem_get_info(dev)[0] == free_before
        r, g = ref.cpu().numpy().reshape(-1, 7), got.cpu().numpy().reshape(-1, 7)
        assert (r[:, 3] >= 0).all() and (r != -7).all()
        assert np.array_equal(g, r)
        assert (r[:, 2] > 0).any()  # the residual path (shared-array U sets) was exercised
    p.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    import torch
    dev = torch.device("cuda:0")
    wl = synth.workload_c2()
    p = perch.Perch(0)
    p.setup(wl)
    n_par = 8  # 8 x 640 x 480 x 4 B of z-buffers alone exceed 8 MiB
    plen = torch.zeros(n_par, dtype=torch.int32, device=dev)
    P = torch.zeros(n_par * 4, dtype=torch.int16, device=dev)
    hp = torch.zeros(4, dtype=torch.int32, device=dev)
    h = torch.zeros(16, dtype=torch.int16, device=dev)
    out = torch.zeros(24, dtype=torch.int32, device=dev)
    with pytest.raises(perch.PerchError) as e:
        p.perch_eval_successors_noalloc(P, 1, plen, hp, h, wl.K, out)
    assert e.value.code == perch.PERCH_E_RANGE
    p.close()
