"""CPU oracle of the learned heuristic network -- TEST INFRASTRUCTURE ONLY.

The paper proposes learning-based heuristics for its multi-heuristic search
(Sec. IV-C names discriminative and learning-based methods as further
heuristics; Sec. VI lists learning as future work) but fixes no network. The
network here predicts y = log(1 + edge cost) of one MSGT successor from two
64 x 64 crops centred on the hypothesis (observed depth and parent z-buffer,
NHWC, 2 channels) and a one-hot of (mesh, yaw):

  conv 3x3 2->32 stride 1, ReLU      64 x 64
  conv 3x3 32->64 stride 2, ReLU     32 x 32
  conv 3x3 64->128 stride 2, ReLU    16 x 16
  conv 3x3 128->128 stride 2, ReLU    8 x 8
  flatten (h, w, c) ++ one-hot -> FC 96, ReLU -> FC 1
  loss = mean 0.5 (pred - y)^2

Convolutions pad by 1; output pixel (i, j) of a stride-s layer reads input
rows s*i - 1 .. s*i + 1 and columns s*j - 1 .. s*j + 1. Weights are
[Cout][3][3][Cin] (conv) and [Out][In] (FC). Everything is float64 unless
`bf16=True`, which rounds the network input, every layer's input activations
and the weights to bfloat16 (round to nearest even) the way the GPU kernels
store them, so that only accumulation order separates the two.
"""
from __future__ import annotations

import numpy as np

CONVS = [(2, 32, 1), (32, 64, 2), (64, 128, 2), (128, 128, 2)]
CROP = 64
FC_HIDDEN = 96


def to_bf16(a):
    """Round float arrays to bfloat16 (nearest even), returned as float64."""
    x = np.asarray(a, np.float32).copy()
    u = x.view(np.uint32).astype(np.uint64)
    bias = ((u >> 16) & 1) + 0x7FFF
    r = ((u + bias) >> 16) << 16
    r = np.where(np.isnan(x), u, r)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def param_shapes(n_onehot: int, crop: int = CROP):
    """Shapes of the twelve parameter arrays, in order (w, b per layer)."""
    shapes = []
    for cin, cout, _ in CONVS:
        shapes += [(cout, 3, 3, cin), (cout,)]
    feat = CONVS[-1][1] * (crop // 8) * (crop // 8)
    shapes += [(FC_HIDDEN, feat + n_onehot), (FC_HIDDEN,), (1, FC_HIDDEN), (1,)]
    return shapes


def _pad(x):
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))


def conv_forward(x, w, b, s):
    """x: (N, H, W, Cin), w: (Cout, 3, 3, Cin) -> (N, H/s, W/s, Cout)."""
    n, h, wd, cin = x.shape
    ho, wo = h // s, wd // s
    xp = _pad(x)
    y = np.zeros((n, ho, wo, w.shape[0]))
    for kh in range(3):
        for kw in range(3):
            patch = xp[:, kh:kh + s * ho:s, kw:kw + s * wo:s, :]  # (N, Ho, Wo, Cin)
            y += np.einsum("nijc,oc->nijo", patch, w[:, kh, kw, :])
    return y + b


def conv_backward(x, w, s, dy):
    """Gradients of conv_forward: (dx, dw, db)."""
    n, h, wd, cin = x.shape
    ho, wo = dy.shape[1], dy.shape[2]
    xp = _pad(x)
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for kh in range(3):
        for kw in range(3):
            patch = xp[:, kh:kh + s * ho:s, kw:kw + s * wo:s, :]
            dw[:, kh, kw, :] = np.einsum("nijo,nijc->oc", dy, patch)
            dxp[:, kh:kh + s * ho:s, kw:kw + s * wo:s, :] += np.einsum("nijo,oc->nijc", dy, w[:, kh, kw, :])
    return dxp[:, 1:-1, 1:-1, :], dw, dy.sum((0, 1, 2))


def forward(params, crops, onehot, bf16: bool = False):
    """Predictions (N,) and the cache needed for the backward pass."""
    r = to_bf16 if bf16 else (lambda a: np.asarray(a, np.float64))
    x = r(crops)
    cache = []
    for li, (cin, cout, s) in enumerate(CONVS):
        w, b = r(params[2 * li]), params[2 * li + 1]
        z = conv_forward(x, w, b, s)
        cache.append((x, w, s, z))
        x = r(np.maximum(z, 0.0))
    feat = np.concatenate([x.reshape(x.shape[0], -1), np.asarray(onehot, np.float64).reshape(x.shape[0], -1)], 1)
    w1, b1, w2, b2 = r(params[8]), params[9], r(params[10]), params[11]
    z1 = feat @ w1.T + b1
    h1 = r(np.maximum(z1, 0.0))
    pred = (h1 @ w2.T + b2)[:, 0]
    return pred, (cache, feat, z1, h1, w1, w2)


def loss_and_grads(params, crops, onehot, target, bf16: bool = False):
    """Mean 0.5 (pred - y)^2 and its gradient for every parameter (float64)."""
    pred, (cache, feat, z1, h1, w1, w2) = forward(params, crops, onehot, bf16)
    n = pred.shape[0]
    err = pred - np.asarray(target, np.float64)
    loss = 0.5 * float(np.mean(err ** 2))
    dpred = (err / n)[:, None]
    grads = [None] * len(params)
    grads[10] = dpred.T @ h1
    grads[11] = dpred.sum(0)
    dh1 = dpred @ w2
    dz1 = dh1 * (z1 > 0)
    grads[8] = dz1.T @ feat
    grads[9] = dz1.sum(0)
    dfeat = dz1 @ w1
    nconv = len(CONVS)
    last = cache[-1][3]
    dx = dfeat[:, :last.size // n].reshape(last.shape)
    for li in range(nconv - 1, -1, -1):
        x, w, s, z = cache[li]
        dz = dx * (z > 0)
        dx, dw, db = conv_backward(x, w, s, dz)
        grads[2 * li], grads[2 * li + 1] = dw, db
    return loss, grads, pred


def grad_magnitudes(params, crops, onehot, target, bf16: bool = False):
    """Scales of the rounding error of every gradient element of
    loss_and_grads, as (sums, rss):
      sums: the sum of the absolute values of the terms the element adds up
            (the same contractions taken on |a| |b|, with the forward pass's
            ReLU masks); a relative perturbation e of every term moves the
            element by at most e * sum, whatever the summation order;
      rss:  the root of the sum of the squared terms; independent relative
            roundings e of the terms move it by about e * rss (a random
            walk), which is what a bfloat16 rounding of each stored operand
            does."""
    pred, (cache, feat, z1, h1, w1, w2) = forward(params, crops, onehot, bf16)
    n = pred.shape[0]
    err = (pred - np.asarray(target, np.float64)) / n
    dpred = err[:, None]
    sums, sq = [None] * len(params), [None] * len(params)
    a = np.abs(dpred)
    sums[10], sq[10] = a.T @ np.abs(h1), (a * a).T @ (h1 * h1)
    sums[11], sq[11] = a.sum(0), (a * a).sum(0)
    dz1 = (dpred @ w2) * (z1 > 0)
    adz1 = (a @ np.abs(w2)) * (z1 > 0)
    sums[8], sq[8] = adz1.T @ np.abs(feat), (dz1 * dz1).T @ (feat * feat)
    sums[9], sq[9] = adz1.sum(0), (dz1 * dz1).sum(0)
    last = cache[-1][3]
    dx = (dz1 @ w1)[:, :last.size // n].reshape(last.shape)
    adx = (adz1 @ np.abs(w1))[:, :last.size // n].reshape(last.shape)
    for li in range(len(CONVS) - 1, -1, -1):
        x, w, s, z = cache[li]
        dz, adz = dx * (z > 0), adx * (z > 0)
        dx, _, _ = conv_backward(x, w, s, dz)
        adx, sw, sb = conv_backward(np.abs(x), np.abs(w), s, adz)
        _, qw, qb = conv_backward(x * x, w, s, dz * dz)
        sums[2 * li], sums[2 * li + 1] = sw, sb
        sq[2 * li], sq[2 * li + 1] = qw, qb
    return sums, [np.sqrt(q) for q in sq]


# ---------------------------------------------------------------------------
# network input: two crops centred on the projected hypothesis
# ---------------------------------------------------------------------------
MISSING = -4.0
CLAMP = 3.0
SCALE = 10.0  # per metre


def crop_centre(cam, mesh, grid, o):
    """Projection of the hypothesis' reference point (x, y, mid-height of
    V(O)) into the image, in float64: (centre column, centre row, z_ref).
    The centre pixel is floor(u + 0.5), floor(v + 0.5)."""
    T = np.asarray(cam.T_wc, np.float32).astype(np.float64).reshape(3, 4)
    p = np.array([float(grid.xs[int(o["ix"])]), float(grid.ys[int(o["iy"])]),
                  (float(np.float32(mesh.vol_zlo)) + float(np.float32(mesh.vol_zhi))) * 0.5])
    d = p - T[:, 3]
    # camera point = R^T (p - t), each coordinate summed in the order 0, 1, 2
    xc = (T[0, 0] * d[0] + T[1, 0] * d[1]) + T[2, 0] * d[2]
    yc = (T[0, 1] * d[0] + T[1, 1] * d[1]) + T[2, 1] * d[2]
    zc = (T[0, 2] * d[0] + T[1, 2] * d[1]) + T[2, 2] * d[2]
    fx, fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    cx, cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
    u = fx * (xc / zc) + cx
    v = fy * (yc / zc) + cy
    return int(np.floor(u + 0.5)), int(np.floor(v + 0.5)), zc


def crop_value(d, z_ref):
    """Depth -> network input: clamp((z_ref - d) * 10 / m, -3, 3), rounded to
    float32 then bfloat16; no return (0, +inf, outside the image) -> -4."""
    d = np.asarray(d, np.float64)
    ok = np.isfinite(d) & (d > 0)
    t = np.where(ok, (z_ref - np.where(ok, d, 0.0)) * SCALE, 0.0).astype(np.float32).astype(np.float64)
    t = np.clip(t, -CLAMP, CLAMP)
    return to_bf16(np.where(ok, t, MISSING))


def crops(cam, meshes, grid, depth, parent_z, hyps, crop: int = CROP):
    """(N, crop, crop, 2) float64 network inputs and (N,) one-hot indices
    (mesh * n_yaw + iyaw): channel 0 is the observed depth, channel 1 the
    parent's z-buffer (+inf where empty). ``parent_z`` is one (H, W) array or
    a list with one per hypothesis."""
    H, W = depth.shape
    out = np.empty((len(hyps), crop, crop, 2))
    idx = np.empty(len(hyps), np.int64)
    for n, o in enumerate(hyps):
        pz = parent_z if isinstance(parent_z, np.ndarray) and parent_z.ndim == 2 else parent_z[n]
        cu, cv, zr = crop_centre(cam, meshes[int(o["mesh"])], grid, o)
        r = np.arange(crop) + cv - crop // 2
        c = np.arange(crop) + cu - crop // 2
        inside = ((r >= 0) & (r < H))[:, None] & ((c >= 0) & (c < W))[None, :]
        rr, cc = np.clip(r, 0, H - 1), np.clip(c, 0, W - 1)
        for ch, img in enumerate((depth, pz)):
            vals = np.asarray(img, np.float64)[rr[:, None], cc[None, :]]
            out[n, :, :, ch] = np.where(inside, crop_value(vals, zr), MISSING)
        idx[n] = int(o["mesh"]) * grid.n_yaw + int(o["iyaw"])
    return out, idx


def onehot(idx, n_onehot: int):
    a = np.zeros((len(idx), n_onehot))
    a[np.arange(len(idx)), idx] = 1.0
    return a


def target(recs):
    """Training target log(1 + dJr + dJo + residual) of edge-cost records."""
    r = np.asarray(recs, np.int64)
    return np.log1p((r[:, 0] + r[:, 1] + r[:, 2]).astype(np.float64))
