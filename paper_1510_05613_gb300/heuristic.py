"""Training data and training loop of the learned heuristic.

The network (its kernels: csrc/perch_cnn.cu) regresses y = log(1 + dJr + dJo
+ residual) of one MSGT successor (Eq. (4) edge cost, Sec. IV-A). Labels are
the exact edge costs of the GPU evaluator; inputs are the library's crops;
training steps are the library's forward, backward and Adam kernels. Nothing
here computes a cost or a gradient: this module only draws which successors
to label and in which order to show them.

Training pairs: seeded scenes (2-5 objects of the eight uneven meshes, the
640x480 camera, 2 cm x 16-yaw grid, objects off the grid by up to half a step
as real objects are); for each scene a seeded random order of
its ground truth gives parents at every level 0..K-1; each parent gets
hypotheses of its remaining types, half near the ground truth (grid offsets
within +-3 cells, yaw within +-2 steps) and half uniform over the grid.
Successors that violate the monotone constraint (Eq. (3)) are dropped.
"""
from __future__ import annotations

import time

import numpy as np

from . import perch, synth

CONVS = [(2, 32), (32, 64), (64, 128), (128, 128)]
HIDDEN = 96
FEAT = 128 * 8 * 8
TRAIN_SEED_BASE = 7000
TEST_SEED_BASE = 9000


def param_shapes(n_onehot: int):
    """Shapes of the parameter arrays in the library's packed order."""
    shapes = []
    for cin, cout in CONVS:
        shapes += [(cout, 3, 3, cin), (cout,)]
    return shapes + [(HIDDEN, FEAT + n_onehot), (HIDDEN,), (1, HIDDEN), (1,)]


def new_network(n_onehot: int, max_batch: int = 256, seed: int = 0, stream=None) -> perch.PerchCNN:
    """A network with seeded He-normal weights and zero biases."""
    net = perch.PerchCNN(n_onehot, max_batch, stream=stream)
    net.perch_cnn_set_params(synth.he_normal(param_shapes(n_onehot), seed))
    return net


def training_scenes(n: int, grid=None, k_range=(2, 5), first: int = 0, off_grid: float = 1.0):
    return synth.workloads_c5(n, grid=grid, k_range=k_range, seed_base=TRAIN_SEED_BASE, first=first,
                              off_grid=off_grid)


def test_scenes(n: int, grid=None, K: int = 5, first: int = 0, off_grid: float = 1.0):
    return synth.workloads_c5(n, grid=grid, k_range=(K, K), seed_base=TEST_SEED_BASE, first=first,
                              off_grid=off_grid)


def _hypotheses(rng, grid, remaining_gt, n_near: int, n_uniform: int):
    """Hypotheses for one parent: near the remaining ground-truth objects and
    uniform over their types."""
    out = np.zeros(n_near + n_uniform, perch.OBJ)
    k = len(remaining_gt)
    pick = rng.integers(0, k, n_near)
    g = remaining_gt[pick]
    out["mesh"][:n_near] = g["mesh"]
    out["ix"][:n_near] = np.clip(g["ix"].astype(np.int64) + rng.integers(-3, 4, n_near), 0, grid.nx - 1)
    out["iy"][:n_near] = np.clip(g["iy"].astype(np.int64) + rng.integers(-3, 4, n_near), 0, grid.ny - 1)
    out["iyaw"][:n_near] = (g["iyaw"].astype(np.int64) + rng.integers(-2, 3, n_near)) % grid.n_yaw
    types = np.unique(remaining_gt["mesh"])
    out["mesh"][n_near:] = types[rng.integers(0, len(types), n_uniform)]
    out["ix"][n_near:] = rng.integers(0, grid.nx, n_uniform)
    out["iy"][n_near:] = rng.integers(0, grid.ny, n_uniform)
    out["iyaw"][n_near:] = rng.integers(0, grid.n_yaw, n_uniform)
    return out


def make_dataset(p: perch.Perch, scenes, scene_ids, per_parent: int = 1024, seed: int = 0, group: int = 16):
    """Labelled pairs from the scenes (already set in context `p` under
    scene_ids). Returns device tensors (crops bf16 (n, 64, 64, 2), one-hot
    indices int32 (n,), targets float32 (n,)) and host statistics."""
    import torch
    rng = np.random.default_rng(seed)
    crops, onehots, targets = [], [], []
    n_eval = n_valid = 0
    t0 = time.perf_counter()
    for g0 in range(0, len(scenes), group):
        parents, pscene, pK, hp, hyps = [], [], [], [], []
        for wl, sid in zip(scenes[g0:g0 + group], scene_ids[g0:g0 + group]):
            order = wl.gt[rng.permutation(wl.K)]
            for j in range(wl.K):
                h = _hypotheses(rng, wl.grid, order[j:], per_parent // 2, per_parent - per_parent // 2)
                hp.append(np.full(len(h), len(parents), np.int32))
                hyps.append(h)
                parents.append(order[:j])
                pscene.append(sid)
                pK.append(wl.K)
        hp, hyps = np.concatenate(hp), np.concatenate(hyps)
        recs = perch.records(p.perch_eval_successors_multi(parents, pscene, pK, hp, hyps))
        valid = recs[:, 3] == 0
        n_eval += len(hyps)
        n_valid += int(valid.sum())
        c, o = p.perch_cnn_crops(parents, hp[valid], hyps[valid], parent_scene=pscene)
        crops.append(c)
        onehots.append(o)
        targets.append(torch.tensor(np.log1p(recs[valid, :3].sum(1).astype(np.float64)), dtype=torch.float32,
                                    device="cuda"))
    crops, onehots, targets = torch.cat(crops), torch.cat(onehots), torch.cat(targets)
    torch.cuda.synchronize()
    return (crops, onehots, targets), {"evaluated": n_eval, "pairs": n_valid,
                                       "seconds": time.perf_counter() - t0}


def train(net: perch.PerchCNN, data, epochs: int = 2, batch: int = 256, lr: float = 1e-3, seed: int = 0,
          lr_final: float = 1e-4, stream=None):
    """Adam on shuffled batches (the last partial batch of an epoch is
    dropped); learning rate decays geometrically from lr to lr_final. Returns
    per-step losses (host) and the seconds spent. ``stream``: the torch stream
    the network was created on (batch gathers are ordered on it)."""
    import torch
    crops, onehot, target = data
    n = crops.shape[0]
    steps_per_epoch = n // batch
    total = steps_per_epoch * epochs
    if total < 1:
        raise ValueError("fewer pairs than one batch")
    losses = torch.zeros(total, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cpu")
    gen.manual_seed(seed)
    stream = stream or torch.cuda.current_stream()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = 0
    with torch.cuda.stream(stream):
        for _ in range(epochs):
            perm = torch.randperm(n, generator=gen).cuda()
            for b in range(steps_per_epoch):
                idx = perm[b * batch:(b + 1) * batch]
                cb, ob, tb = crops[idx], onehot[idx], target[idx]
                lr_k = lr * (lr_final / lr) ** (k / max(1, total - 1))
                net.perch_cnn_train_step(cb, ob, tb, lr_k, losses[k:k + 1])
                k += 1
    torch.cuda.synchronize()
    return losses.cpu().numpy(), time.perf_counter() - t0


def evaluate(net: perch.PerchCNN, data):
    """Held-out regression quality: mean squared error, Pearson and Spearman
    correlation between predictions and targets."""
    crops, onehot, target = data
    pred = net.perch_cnn_forward(crops, onehot).cpu().numpy().astype(np.float64)
    y = target.cpu().numpy().astype(np.float64)
    rank = lambda a: np.argsort(np.argsort(a)).astype(np.float64)
    return {"mse": float(np.mean((pred - y) ** 2)), "var": float(np.var(y)),
            "pearson": float(np.corrcoef(pred, y)[0, 1]), "spearman": float(np.corrcoef(rank(pred), rank(y))[0, 1]),
            "n": int(len(y))}


def setup_scenes(p: perch.Perch, scenes, first_id: int = 0):
    """Load meshes, grid and the first scene's observation into `p`, then every
    scene under ids first_id, first_id + 1, ...; returns the ids."""
    wl0 = scenes[0]
    if first_id == 0:
        p.setup(wl0)
    ids = []
    for k, wl in enumerate(scenes):
        sid = first_id + k
        if sid > 0:
            p.perch_set_scene(sid, wl.depth)
        ids.append(sid)
    return ids
