"""Pins of the oracle's student training pieces (FP64)."""
import math

import numpy as np

import synth
from oracle import schedule as S
from oracle import student as OS
from oracle import unet as OU

import torch


def tiny():
    return synth.level(levels=2, channels=(8, 8), in_ch=1, out_ch=1, window=16, gn_groups=4)


def test_torch_forward_equals_numpy_oracle():
    lv = synth.level(levels=3, channels=(8, 16, 16), in_ch=1, out_ch=1, window=16, gn_groups=4)
    w = synth.weights([s for _, s in OU.param_shapes(lv)], 0, 0)
    x = synth.window_batch(2, 1, 16, seed=3).astype(np.float64)
    ref = OU.forward(lv, OU.unpack(lv, w), x)
    with torch.no_grad():
        got = OS.forward_torch(lv, OS._params(lv, w, False), torch.as_tensor(x)).numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_gradient_matches_central_differences():
    lv = tiny()
    w = synth.weights([s for _, s in OU.param_shapes(lv)], 1, 0).astype(np.float64)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 16, 16)) * 3.0
    t = rng.standard_normal((2, 16, 16)) * 0.3
    sigma = 0.8
    loss, g = OS.loss_and_grad(lv, w, x, t, sigma)
    assert math.isfinite(loss)
    idx = rng.choice(w.size, size=24, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (OS.loss_only(lv, wp, x, t, sigma) - OS.loss_only(lv, wm, x, t, sigma)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_adamw_step_by_hand():
    w, m, v = np.array([1.0]), np.array([0.0]), np.array([0.0])
    g = np.array([0.5])
    w1, m1, v1 = OS.adamw(w, g, m, v, 1, lr=0.1, wd=0.01)
    # m = 0.05, v = 0.00025, mh = 0.5, vh = 0.25 -> step 0.5 / (0.5 + 1e-8)
    assert abs(m1[0] - 0.05) < 1e-15 and abs(v1[0] - 0.001 * 0.25) < 1e-15
    expect = 1.0 - 0.1 * (0.5 / (0.5 + 1e-8) + 0.01 * 1.0)
    assert abs(w1[0] - expect) < 1e-15


def test_side_channels_enter_unscaled_and_state_only_through_channel_zero():
    # a 3-channel student whose in-conv ignores channel 0 and reads channel 1
    # with the weights of a 1-channel network: D(x; sigma) = c_skip x_0 +
    # c_out F_1(x_1) exactly when the side channels reach S unscaled
    lv1 = tiny()
    lv3 = dict(lv1, in_ch=3)
    w1 = synth.weights([s for _, s in OU.param_shapes(lv1)], 2, 0).astype(np.float64)
    shapes1 = OU.param_shapes(lv1)
    shapes3 = OU.param_shapes(lv3)
    parts, o = [], 0
    for (n1, s1), (n3, s3) in zip(shapes1, shapes3):
        k = int(np.prod(s1))
        a = w1[o:o + k].reshape(s1)
        o += k
        if n1 == "in_conv":
            b = np.zeros(s3)
            b[:, 1:2] = a
            a = b
        parts.append(a.reshape(-1))
    w3 = np.concatenate(parts)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, 3, 16, 16))
    sigma = 2.5
    c_skip, c_out, c_in = S.edm_coeffs(sigma, float(lv1["sigma_data"]))
    with torch.no_grad():
        d3 = OS._denoise(lv3, OS._params(lv3, w3, False), x, sigma).numpy()[:, 0]
        f1 = OS.forward_torch(lv1, OS._params(lv1, w1, False), torch.as_tensor(x[:, 1:2])).numpy()[:, 0]
    ref = c_skip * x[:, 0] + c_out * f1
    assert np.max(np.abs(d3 - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_gradient_with_side_channels_matches_central_differences():
    lv = dict(tiny(), in_ch=3)
    w = synth.weights([s for _, s in OU.param_shapes(lv)], 4, 0).astype(np.float64)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 16, 16))
    t = rng.standard_normal((2, 16, 16)) * 0.3
    sigma = 80.0
    loss, g = OS.loss_and_grad(lv, w, x, t, sigma)
    assert math.isfinite(loss)
    h = 1e-6
    for i in rng.choice(w.size, size=16, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (OS.loss_only(lv, wp, x, t, sigma) - OS.loss_only(lv, wm, x, t, sigma)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9, (i, fd, g[i])

