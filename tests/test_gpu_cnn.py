"""GPU parity of the learned heuristic's network against its CPU oracle.

Crops are compared bit for bit (both sides follow the same double-precision
centre and float/bfloat16 rounding). The network's forward and backward pass
run in bfloat16 with FP32 accumulation and bfloat16 gradients between layers,
against the oracle in float64 with the same bfloat16 rounding of inputs,
activations and weights: predictions within 2e-2 (absolute, on targets of
size ~1) and the loss within 1e-2 relative. Gradients are compared element by
element: the oracle's backward pass is given the GPU's own prediction error
(its target shifted by pred_gpu - pred_oracle), so only the backward pass
separates them. The GPU stores every gradient between layers in bfloat16
(relative rounding 2^-9 per element) and the deepest weight gradient sits
six such roundings below the loss; FP32 accumulation adds n 2^-24 relative
per term. With S the root of the sum of the squared terms an element adds up
(oracle.cnn.grad_magnitudes), independent roundings move it like a random
walk over the fan-in, so each element must satisfy
    |g - e| <= 8 2^-9 S + 2^-7 |e|      (8 standard widths).
Exceptions have a known cause: where a pre-activation lies within the two
sides' accumulation difference of zero, their ReLU masks differ, and that
one position adds or drops a whole term, in the forward pass (an activation
feeding every weight gradient of the next layer) or in the backward pass (a
gradient feeding every weight gradient of its output channel). Measured:
0.17% of conv4's 147k weight gradients; an FC1 gradient with one term
doubled. So in a tensor of 1000 or more elements at most 0.5% may exceed the
bound, and in a smaller tensor at most one element. A wrong sign or index on
a slice of a tensor (one channel of 128 is 0.78%, one tap of nine 11%) moves
its elements by about |e| or S and fails it.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import cnn
from paper_1510_05613_gb300 import perch, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    wl = synth.workload_c1()
    p = perch.Perch(0)
    p.setup(wl)
    return wl, p, oracle.World.of(wl)


def _hyps_c1(wl, n, seed):
    rng = np.random.default_rng(seed)
    all_h = synth.all_hypotheses(wl.grid, [0, 1])
    return all_h[rng.choice(len(all_h), n, replace=False)]


def _crops_both(wl, p, w, parent, hyps):
    crops, onehot = p.perch_cnn_crops([parent], np.zeros(len(hyps), np.int32), hyps)
    pz, _ = oracle.render(w, parent)
    exp, idx = cnn.crops(wl.cam, wl.meshes, wl.grid, wl.depth, pz, hyps)
    return crops, onehot, exp, idx


def test_crops_bit_exact(c1):
    wl, p, w = c1
    hyps = _hyps_c1(wl, 96, 1)
    for parent in (wl.gt[:0], wl.gt[:1]):
        crops, onehot, exp, idx = _crops_both(wl, p, w, parent, hyps)
        got = crops.float().cpu().numpy().astype(np.float64)
        assert np.array_equal(onehot.cpu().numpy(), idx)
        bad = np.argwhere(got != exp)
        assert bad.size == 0, (bad[:5], got[tuple(bad[0])], exp[tuple(bad[0])])
        assert (exp[..., 0] > -4).any() and (exp[..., 0] == -4).any()


def _params(n_onehot, seed):
    return [a.astype(np.float64) for a in synth.he_normal(cnn.param_shapes(n_onehot), seed)]


def _net_with(params, n_onehot, max_batch=64):
    net = perch.PerchCNN(n_onehot, max_batch)
    net.perch_cnn_set_params(params)
    return net


def test_gradients_match_oracle(c1):
    wl, p, w = c1
    n_onehot = len(wl.meshes) * wl.grid.n_yaw
    hyps = _hyps_c1(wl, 32, 2)
    crops, onehot, x, idx = _crops_both(wl, p, w, wl.gt[:1], hyps)
    params = _params(n_onehot, 3)
    rng = np.random.default_rng(4)
    params[9] += 0.1 * rng.standard_normal(params[9].shape)  # some FC biases on
    y = rng.uniform(0.0, 4.0, 32)
    net = _net_with(params, n_onehot)
    target = torch.tensor(y, dtype=torch.float32, device="cuda")
    g, loss, pred = net.perch_cnn_gradients(crops, onehot, target)
    # the parameters the network holds: round-trip of the set values
    assert np.array_equal(net.perch_cnn_get_params(), np.concatenate([a.astype(np.float32).ravel() for a in params]))
    oh = cnn.onehot(idx, n_onehot)
    el, _, ep = cnn.loss_and_grads(params, x, oh, y, bf16=True)
    assert np.max(np.abs(pred - ep)) < 2e-2
    assert abs(loss - el) <= 1e-2 * el
    # the oracle's backward pass from the GPU's prediction error
    y_adj = y - (pred.astype(np.float64) - ep)
    _, eg, _ = cnn.loss_and_grads(params, x, oh, y_adj, bf16=True)
    _, rss = cnn.grad_magnitudes(params, x, oh, y_adj, bf16=True)
    off, n_el, n_stat = 0, 0, 0
    for k, (e, r) in enumerate(zip(eg, rss)):
        got = g[off:off + e.size].reshape(e.shape).astype(np.float64)
        off += e.size
        err = np.abs(got - e)
        stat = 8 * 2.0 ** -9 * r + 2.0 ** -7 * np.abs(e) + 1e-30
        ok = err <= stat
        worst = np.unravel_index(np.argmax(err / stat), e.shape)
        allowed = int(0.005 * e.size) if e.size >= 1000 else 1
        assert int((~ok).sum()) <= allowed, (k, ok.mean(), worst, got[worst], e[worst], r[worst])
        n_el += e.size
        n_stat += int(ok.sum())
    assert off == net.n_params == n_el and n_stat >= 0.995 * n_el


def test_forward_ragged_batch_matches_oracle(c1):
    wl, p, w = c1
    n_onehot = len(wl.meshes) * wl.grid.n_yaw
    hyps = _hyps_c1(wl, 77, 5)  # not a multiple of 32, more than max_batch: two chunks
    crops, onehot, x, idx = _crops_both(wl, p, w, wl.gt[1:], hyps)
    params = _params(n_onehot, 6)
    net = _net_with(params, n_onehot, max_batch=64)
    pred = net.perch_cnn_forward(crops, onehot).cpu().numpy()
    ep, _ = cnn.forward(params, x, cnn.onehot(idx, n_onehot), bf16=True)
    assert np.max(np.abs(pred - ep)) < 2e-2 * max(1.0, np.max(np.abs(ep)))
    assert np.all(np.isfinite(pred))


def test_adam_first_step_moves_by_lr_times_sign(c1):
    """Adam's first step with zero moments is lr * g / (|g| + eps): every
    parameter whose gradient is clearly non-zero moves by -lr sign(g)."""
    wl, p, w = c1
    n_onehot = len(wl.meshes) * wl.grid.n_yaw
    hyps = _hyps_c1(wl, 32, 7)
    crops, onehot, x, idx = _crops_both(wl, p, w, wl.gt[:0], hyps)
    params = _params(n_onehot, 8)
    net = _net_with(params, n_onehot)
    y = np.random.default_rng(9).uniform(0.0, 4.0, 32)
    _, eg, _ = cnn.loss_and_grads(params, x, cnn.onehot(idx, n_onehot), y, bf16=True)
    target = torch.tensor(y, dtype=torch.float32, device="cuda")
    lr = 1e-3
    net.perch_cnn_train_step(crops, onehot, target, lr)
    torch.cuda.synchronize()
    after = net.perch_cnn_get_params().astype(np.float64)
    before = np.concatenate([a.astype(np.float32).ravel() for a in params]).astype(np.float64)
    g = np.concatenate([e.ravel() for e in eg])
    clear = np.abs(g) > 0.1 * np.sqrt(np.mean(g ** 2))  # away from where bfloat16 noise decides the sign
    step = after - before
    assert clear.sum() > 1000
    assert np.mean(np.abs(step[clear] + lr * np.sign(g[clear])) < 0.05 * lr) > 0.99
    assert np.max(np.abs(step)) <= lr * 1.001


def test_training_reduces_the_loss(c1):
    wl, p, w = c1
    n_onehot = len(wl.meshes) * wl.grid.n_yaw
    hyps = _hyps_c1(wl, 256, 10)
    parents = [wl.gt[:0], wl.gt[:1], wl.gt[1:]]
    hp = np.arange(256, dtype=np.int32) % 3
    recs = perch.records(p.perch_eval_successors(parents, hp, hyps, 2))
    valid = recs[:, 3] == 0
    crops, onehot = p.perch_cnn_crops(parents, hp, hyps)
    keep = torch.from_numpy(np.nonzero(valid)[0][:224]).cuda()
    assert keep.numel() == 224
    crops, onehot = crops[keep].contiguous(), onehot[keep].contiguous()
    y = np.log1p(recs[valid][:224, :3].sum(1).astype(np.float64))
    target = torch.tensor(y, dtype=torch.float32, device="cuda")
    net = _net_with(_params(n_onehot, 11), n_onehot, max_batch=224)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    hist = []
    for step in range(60):
        net.perch_cnn_train_step(crops, onehot, target, 1e-3, loss)
        torch.cuda.synchronize()
        hist.append(float(loss.item()))
    assert all(np.isfinite(hist))
    assert hist[-1] < 0.3 * hist[0], hist[::10]


@pytest.mark.parametrize("n,max_batch", [(77, 64), (256, 256)])
def test_tcgen05_forward_matches_mma_sync_and_oracle(c1, n, max_batch):
    """The forward 3x3 convolutions 2-4 on tcgen05 (FP32 accumulator in tensor
    memory) against the mma.sync path and the oracle, on a ragged batch (row
    tiles of 128 that end inside the batch) and a full one. Both tensor paths
    round the same FP32 sums to bfloat16 after bias and ReLU, in different
    summation orders: predictions agree within the bfloat16 tolerance of the
    oracle comparison, and no bounded wait of the tcgen05 kernel gives up."""
    wl, p, w = c1
    n_onehot = len(wl.meshes) * wl.grid.n_yaw
    hyps = _hyps_c1(wl, n, 12 + n)
    crops, onehot, x, idx = _crops_both(wl, p, w, wl.gt[:1], hyps)
    params = _params(n_onehot, 13)
    net = _net_with(params, n_onehot, max_batch=max_batch)
    ref = net.perch_cnn_forward(crops, onehot).cpu().numpy()
    net.perch_cnn_set_tensor_path(1)
    got = net.perch_cnn_forward(crops, onehot).cpu().numpy()
    assert net.perch_cnn_tensor_status() == (1, 0)
    ep, _ = cnn.forward(params, x, cnn.onehot(idx, n_onehot), bf16=True)
    scale = max(1.0, float(np.max(np.abs(ep))))
    assert np.all(np.isfinite(got))
    assert np.max(np.abs(got - ep)) < 2e-2 * scale
    assert np.max(np.abs(got - ref)) < 2e-2 * scale
    with pytest.raises(perch.PerchError):
        net.perch_cnn_set_tensor_path(2)
