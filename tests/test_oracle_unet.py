"""Pin of the oracle UNet against torch.nn.functional in FP64 (library routines)."""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as TF

import synth
from oracle import unet as U


def torch_forward(lv, p, x, y=None):
    """The same network written with torch.nn.functional layers (FP64);
    y: per-window conditioning vectors embedded by F.linear as a bias."""
    G = lv["gn_groups"]
    t = {k: torch.from_numpy(v) for k, v in p.items()}

    def gn(h):
        return TF.group_norm(h, G, eps=1e-5)

    def conv(h, w):
        return TF.conv2d(h, w, padding=w.shape[-1] // 2)

    def rb(h, name):
        a = conv(TF.silu(gn(h)), t[name + ".conv1"])
        a = conv(TF.silu(gn(a)), t[name + ".conv2"])
        return a + (conv(h, t[name + ".skip"]) if name + ".skip" in t else h)

    h = conv(torch.from_numpy(x), t["in_conv"])
    if y is not None:
        h = h + TF.linear(torch.from_numpy(y), t["cond_embed"][:, :, 0, 0])[:, :, None, None]
    skips = []
    L = lv["levels"]
    for l in range(L):
        h = rb(h, f"enc{l}")
        skips.append(h)
        if l < L - 1:
            h = TF.avg_pool2d(h, 2)
    if lv["attn_at_bottom"]:
        B, C, Hh, Ww = h.shape
        heads = lv["attn_heads"]
        d = C // heads
        qkv = conv(gn(h), t["attn.qkv"]).reshape(B, 3, heads, d, Hh * Ww)
        q, k, v = qkv[:, 0].transpose(-1, -2), qkv[:, 1].transpose(-1, -2), qkv[:, 2].transpose(-1, -2)
        a = torch.softmax(q @ k.transpose(-1, -2) / math.sqrt(d), dim=-1)
        o = (a @ v).transpose(-1, -2).reshape(B, C, Hh, Ww)
        h = h + conv(o, t["attn.proj"])
    h = rb(h, "mid")
    for l in range(L - 2, -1, -1):
        h = torch.cat([TF.interpolate(h, scale_factor=2, mode="nearest"), skips[l]], dim=1)
        h = rb(h, f"dec{l}")
    return conv(TF.silu(gn(h)), t["out_conv"]).numpy()


@pytest.mark.parametrize("lv", [
    synth.config1_stack()["level"][0],
    synth.small_hier_stack()["level"][1],
    synth.level(levels=3, channels=(8, 16, 16), in_ch=2, attn_at_bottom=1, attn_heads=2, window=16),
])
def test_unet_matches_torch_functional(lv):
    shapes = [s for _, s in U.param_shapes(lv)]
    w = synth.weights(shapes, 0, 0)
    p = U.unpack(lv, w)
    x = synth.window_batch(3, lv["in_ch"], lv["window"], seed=1, scale=2.0).astype(np.float64)
    got = U.forward(lv, p, x)
    ref = torch_forward(lv, p, x)
    assert got.shape == (3, lv["out_ch"], lv["window"], lv["window"])
    assert np.max(np.abs(got - ref)) <= 1e-11 * max(1.0, np.max(np.abs(ref)))


def test_param_count_and_flops_config1():
    lv = synth.config1_stack()["level"][0]
    names = [n for n, _ in U.param_shapes(lv)]
    assert names == ["in_conv", "enc0.conv1", "enc0.conv2", "enc1.conv1", "enc1.conv2",
                     "mid.conv1", "mid.conv2", "dec0.conv1", "dec0.conv2", "dec0.skip", "out_conv"]
    # 29.95 MFLOP per 32x32 window (convolutions, 2 FLOP per MAC)
    assert abs(U.flops_per_window(lv) / 1e6 - 29.95) < 0.01


def test_flops_config2():
    st = synth.config2_stack()
    fine = U.flops_per_window(st["level"][1]) / 1e9
    coarse = U.flops_per_window(st["level"][0]) / 1e9
    assert abs(fine - 22.0) < 0.1 and abs(coarse - 14.67) < 0.1


def test_conv_is_cross_correlation():
    # a kernel with a single 1 at the top-left tap shifts the image by (+1, +1)
    x = np.arange(16, dtype=np.float64).reshape(1, 1, 4, 4)
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 0, 0] = 1.0
    y = U.conv(x, w)[0, 0]
    assert y[1, 1] == x[0, 0, 0, 0] and y[0, 0] == 0.0 and y[3, 3] == x[0, 0, 2, 2]


def test_upsampled_branch_phase_identity():
    # The identity the tensor-core path uses for decoder blocks: a 3x3
    # convolution of [nearest-up2(a), b] equals the 3x3 convolution of b plus,
    # for each output phase (py, px), a 2x2 convolution of a at its own
    # resolution whose taps sum the 3x3 taps reading the same pixel of a
    # (input rows floor((2Y + py + dy) / 2) = Y + py - 1 + ty); and the 1x1
    # shortcut of the concat equals up2(W_a a) + W_b b.
    rng = np.random.default_rng(11)
    Ca, Cb, Co, h = 3, 2, 4, 5
    a = rng.standard_normal((1, Ca, h, h))
    b = rng.standard_normal((1, Cb, 2 * h, 2 * h))
    w = rng.standard_normal((Co, Ca + Cb, 3, 3))
    wsk = rng.standard_normal((Co, Ca + Cb, 1, 1))
    cat = np.concatenate([U.up2(a), b], axis=1)
    ref = U.conv(cat, w)
    out = U.conv(b, w[:, Ca:])
    ap = np.pad(a, ((0, 0), (0, 0), (1, 1), (1, 1)))
    for py in range(2):
        for px in range(2):
            wp = np.zeros((Co, Ca, 2, 2))
            for ky in range(3):
                for kx in range(3):
                    ty = (py + ky - 1) // 2 - (py - 1)
                    tx = (px + kx - 1) // 2 - (px - 1)
                    wp[:, :, ty, tx] += w[:, :Ca, ky, kx]
            ph = np.zeros((1, Co, h, h))
            for ty in range(2):
                for tx in range(2):
                    oy, ox = py - 1 + ty, px - 1 + tx
                    ph += np.einsum("oc,bchw->bohw", wp[:, :, ty, tx],
                                    ap[:, :, 1 + oy:1 + oy + h, 1 + ox:1 + ox + h])
            out[:, :, py::2, px::2] += ph
    assert np.allclose(out, ref, rtol=0, atol=1e-12)
    sk_ref = U.conv(cat, wsk)
    sk = U.up2(U.conv(a, wsk[:, :Ca])) + U.conv(b, wsk[:, Ca:])
    assert np.allclose(sk, sk_ref, rtol=0, atol=1e-12)


def test_conditioning_bias_matches_torch_linear():
    # the per-window conditioning vector enters as E y added after the in-conv
    st = synth.conditioned(synth.config1_stack(), dim=4)
    lv = st["level"][0]
    p = U.unpack(lv, synth.weights([s for _, s in U.param_shapes(lv)], 0, 0))
    x = synth.window_batch(3, 1, 32, seed=2).astype(np.float64)
    y = np.random.default_rng(0).standard_normal((3, 4))
    got = U.forward(lv, p, x, y)
    ref = np.asarray(torch_forward(lv, p, x, y))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # and it changes the output (a dropped bias would not)
    assert np.max(np.abs(got - U.forward(lv, p, x))) > 1e-3 * np.max(np.abs(ref))
