"""Pins of the learned heuristic's CPU oracle (network of the multi-heuristic
search, Sec. IV-C): bfloat16 rounding against torch's conversion, the
convolution against a brute-force loop and against torch's conv2d, every
gradient against torch autograd (float64) and against central finite
differences, a closed-form loss, and the crop geometry on a camera looking
straight down."""
import math

import numpy as np
import pytest
import torch

from oracle import cnn
from paper_1510_05613_gb300 import synth


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0, -0.0, 3.0e38])])
    x = x.astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.to_bf16(x), want)


def _brute_conv(x, w, b, s):
    n, h, wd, cin = x.shape
    cout = w.shape[0]
    y = np.zeros((n, h // s, wd // s, cout))
    for a in range(n):
        for i in range(h // s):
            for j in range(wd // s):
                for o in range(cout):
                    acc = b[o]
                    for kh in range(3):
                        for kw in range(3):
                            r, c = s * i - 1 + kh, s * j - 1 + kw
                            if 0 <= r < h and 0 <= c < wd:
                                acc += float(np.dot(x[a, r, c, :], w[o, kh, kw, :]))
                    y[a, i, j, o] = acc
    return y


@pytest.mark.parametrize("s", [1, 2])
def test_conv_matches_brute_force_and_torch(s):
    rng = np.random.default_rng(s)
    x = rng.standard_normal((2, 6, 8, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv_forward(x, w, b, s)
    assert np.allclose(y, _brute_conv(x, w, b, s), atol=1e-12)
    yt = torch.nn.functional.conv2d(torch.from_numpy(x).permute(0, 3, 1, 2), torch.from_numpy(w).permute(0, 3, 1, 2),
                                    torch.from_numpy(b), stride=s, padding=1).permute(0, 2, 3, 1).numpy()
    assert np.allclose(y, yt, atol=1e-12)


def _torch_model(params, crops, onehot, target):
    """The same network in torch ops (float64, NCHW), for autograd."""
    ps = [torch.tensor(p, dtype=torch.float64, requires_grad=True) for p in params]
    x = torch.from_numpy(crops).permute(0, 3, 1, 2)
    for li, (_, _, s) in enumerate(cnn.CONVS):
        x = torch.relu(torch.nn.functional.conv2d(x, ps[2 * li].permute(0, 3, 1, 2), ps[2 * li + 1], stride=s,
                                                  padding=1))
    feat = torch.cat([x.permute(0, 2, 3, 1).reshape(x.shape[0], -1), torch.from_numpy(onehot)], 1)
    h = torch.relu(feat @ ps[8].T + ps[9])
    pred = (h @ ps[10].T + ps[11])[:, 0]
    loss = 0.5 * ((pred - torch.from_numpy(target)) ** 2).mean()
    loss.backward()
    return float(loss.detach()), [p.grad.numpy() for p in ps], pred.detach().numpy()


def _tiny(crop=16, n=3, n_onehot=5, seed=4):
    params = [p.astype(np.float64) for p in synth.he_normal(cnn.param_shapes(n_onehot, crop), seed)]
    rng = np.random.default_rng(seed)
    params = [p + 0.05 * rng.standard_normal(p.shape) for p in params]  # non-zero biases too
    x = rng.uniform(-4, 3, (n, crop, crop, 2))
    oh = cnn.onehot(rng.integers(0, n_onehot, n), n_onehot)
    y = rng.uniform(0, 5, n)
    return params, x, oh, y


def test_gradients_match_torch_autograd():
    params, x, oh, y = _tiny()
    loss, grads, pred = cnn.loss_and_grads(params, x, oh, y)
    tl, tg, tp = _torch_model(params, x, oh, y)
    assert math.isclose(loss, tl, rel_tol=1e-12)
    assert np.allclose(pred, tp, atol=1e-12)
    for g, t in zip(grads, tg):
        assert g.shape == t.shape
        assert np.allclose(g, t, rtol=1e-9, atol=1e-12)


def test_gradients_match_finite_differences():
    params, x, oh, y = _tiny(seed=9)
    _, grads, _ = cnn.loss_and_grads(params, x, oh, y)
    rng = np.random.default_rng(1)
    eps = 1e-6
    checked = 0
    for li, p in enumerate(params):
        for _ in range(4):
            i = tuple(int(rng.integers(0, d)) for d in p.shape)
            saved = p[i]
            p[i] = saved + eps
            lp = cnn.loss_and_grads(params, x, oh, y)[0]
            p[i] = saved - eps
            lm = cnn.loss_and_grads(params, x, oh, y)[0]
            p[i] = saved
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - grads[li][i]) <= 1e-6 + 1e-5 * abs(fd), (li, i, fd, grads[li][i])
            checked += 1
    assert checked == 48


def test_loss_closed_form_with_zero_weights():
    params, x, oh, y = _tiny()
    params = [np.zeros_like(p) for p in params]
    params[11][0] = 1.5
    loss, grads, pred = cnn.loss_and_grads(params, x, oh, y)
    assert np.all(pred == 1.5)
    assert math.isclose(loss, 0.5 * np.mean((1.5 - y) ** 2), rel_tol=1e-15)
    assert math.isclose(float(grads[11][0]), float(np.mean(1.5 - y)), rel_tol=1e-12)
    assert all(not g.any() for g in grads[:11])  # every ReLU is off


def test_bf16_mode_only_rounds_inputs_and_weights():
    params, x, oh, y = _tiny(seed=5)
    p16 = [cnn.to_bf16(p) if p.ndim > 1 else p for p in params]
    a = cnn.forward(params, cnn.to_bf16(x), oh, bf16=True)[0]
    b = cnn.forward(p16, cnn.to_bf16(x), oh, bf16=True)[0]
    assert np.array_equal(a, b)
    full = cnn.forward(params, x, oh)[0]
    assert np.max(np.abs(a - full)) < 0.05 * (1 + np.max(np.abs(full)))


def _down_camera(W=64, H=48):
    # straight down from 1 m above (0.1, -0.05): x right = world +x, y down = world -y
    T = np.array([[1, 0, 0, 0.1], [0, -1, 0, -0.05], [0, 0, -1, 1.0]], np.float32)
    return synth.Camera(W, H, 100.0, 100.0, 30.0, 20.0, T)


def test_crop_centre_and_values_on_a_downward_camera():
    cam = _down_camera()
    mesh = synth.Mesh("m", np.zeros((1, 3), np.float32), np.zeros((0, 3), np.int32), 0.02, 0.0, 0.5)
    grid = synth.PoseGrid(np.array([0.1, 0.2], np.float32), np.array([-0.05], np.float32),
                          np.array([[1.0, 0.0]], np.float32))
    # below the camera: centre (cx, cy) = (30, 20), z_ref = 1 - 0.25 = 0.75 (exact in binary)
    o = synth.objs([(0, 0, 0, 0)])
    cu, cv, zr = cnn.crop_centre(cam, mesh, grid, o[0])
    assert (cu, cv) == (30, 20) and zr == 0.75
    # 0.1 m to the right at 0.75 m depth: u = 30 + 100 * 0.1 / 0.75
    cu2, cv2, _ = cnn.crop_centre(cam, mesh, grid, synth.objs([(0, 1, 0, 0)])[0])
    assert (cu2, cv2) == (math.floor(30 + 100 * 0.1 / 0.75 + 0.5), 20)
    depth = np.full((cam.H, cam.W), 0.75, np.float32)
    depth[20, 30] = 0.70  # the centre pixel: 5 cm nearer than z_ref -> 0.5
    depth[21, 30] = 0.0  # no return
    depth[0, 0] = 0.1  # far in front -> clamped to 3
    pz = np.full_like(depth, np.inf)
    x, idx = cnn.crops(cam, [mesh], grid, depth, pz, o, crop=16)
    c0, c1 = x[0, :, :, 0], x[0, :, :, 1]
    assert c0[8, 8] == 0.5
    assert c0[9, 8] == -4.0 and np.all(c1 == -4.0)
    assert c0[8, 9] == 0.0 and c0[7, 7] == 0.0
    # rows 20-8 .. 20+7 and columns 30-8 .. 30+7 are all inside the 64 x 48 image
    assert np.count_nonzero(c0 == -4.0) == 1 and idx[0] == 0
    x2, _ = cnn.crops(cam, [mesh], grid, depth, pz, o, crop=64)
    # crop 64 around (30, 20): columns -2..61 and rows -12..51 -> 2 and 12 + 4 outside
    outside = np.ones((64, 64), bool)
    outside[12:12 + 48, 2:2 + 64] = False
    assert np.all(x2[0, :, :, 0][outside] == -4.0)
    assert x2[0, 12, 2, 0] == 3.0  # depth[0, 0] = 0.1: clamped


def test_target_is_log1p_of_the_edge_cost():
    recs = np.array([[3, 4, 5, 0, 9, 0, 1], [0, 0, 0, 0, 2, 0, 0]], np.int32)
    assert np.allclose(cnn.target(recs), [math.log(13.0), 0.0])
