"""Window denoiser F (oracle): the synthetic ResBlock UNet, FP64.

Test infrastructure (see the package header).

The paper's networks are EDM2+sCM UNets with trained weights (Sec. 5.3,
Table "Hyperparameters", App. F), which are not available; the synthetic
stacks replace them by plain conv UNets of the stated widths.  The reading
fixed for them (everything the stack description leaves open):

* in-conv 3x3 (in_ch -> c0);
* encoder level l = 0..L-1: ResBlock(c_prev -> c_l), then 2x2 average pool
  except after the last level; the ResBlock output before pooling is the
  skip of level l;
* bottom: optional self-attention block, then ResBlock(c_{L-1} -> c_{L-1});
* decoder level l = L-2..0: nearest x2 upsample, channel concat
  [upsampled, skip_l], ResBlock(c_up + c_l -> c_l);
* out: GroupNorm, SiLU, conv 3x3 (c0 -> out_ch).
* ResBlock(x): h = conv1(silu(gn(x))); h = conv2(silu(gn(h)));
  return h + shortcut(x), shortcut = 1x1 conv when channels change, else x.
* Attention block: h = gn(x); [q; k; v] = 1x1 conv (C -> 3C); per head
  (d = C/heads channels, tokens = pixels) softmax(q^T k / sqrt(d)) v;
  x + 1x1 proj (C -> C).
* GroupNorm: gn_groups groups, population variance, eps 1e-5, affine 1/0.
* Zero padding per window (each window is an independent image to Phi,
  App. B "Pretrained diffusion model").  No biases (zero by the reading).
* Conv weights are (C_out, C_in, kh, kw), cross-correlation as in every deep
  learning framework; parameters are declared in the order listed above
  (per ResBlock: conv1, conv2, then shortcut if any; attention: qkv, proj).

Per-window conditioning (App. B "Seeds and initial noise": y_i = Lambda(z, i);
Sec. 5.3 injects such a vector, the climate scalars, alongside the noise
embedding): with cond_dim = D > 0 the network takes a vector y of D values
per window and adds E y, E a (c0, D) linear embedding declared last among
the parameters ("cond_embed"), as a per-channel bias to the in-conv output.

Test denoisers (closed-form pins of the sampler, not networks): 1 = constant
F = 0.5; 2 = identity F = sum of input channels; 3 = local coordinate
F = sum of input channels + u/H - 2 v/H (u row, v column inside the window).

Pins: FP64 agreement with torch.nn.functional (conv2d, group_norm, silu,
avg_pool2d, interpolate, softmax) on the same weights
(tests/test_oracle_unet.py).
"""
from __future__ import annotations

import math

import numpy as np

GN_EPS = 1e-5


def param_shapes(lv: dict):
    """[(name, (C_out, C_in, kh, kw)), ...] in declaration order."""
    L = int(lv["levels"])
    ch = [int(c) for c in lv["channels"]]
    out = [("in_conv", (ch[0], int(lv["in_ch"]), 3, 3))]

    def rb(name, cin, cout):
        out.append((name + ".conv1", (cout, cin, 3, 3)))
        out.append((name + ".conv2", (cout, cout, 3, 3)))
        if cin != cout:
            out.append((name + ".skip", (cout, cin, 1, 1)))

    prev = ch[0]
    for l in range(L):
        rb(f"enc{l}", prev, ch[l])
        prev = ch[l]
    if int(lv.get("attn_at_bottom", 0)):
        C = prev
        out.append(("attn.qkv", (3 * C, C, 1, 1)))
        out.append(("attn.proj", (C, C, 1, 1)))
    rb("mid", prev, prev)
    for l in range(L - 2, -1, -1):
        rb(f"dec{l}", prev + ch[l], ch[l])
        prev = ch[l]
    out.append(("out_conv", (int(lv["out_ch"]), prev, 3, 3)))
    if int(lv.get("cond_dim", 0)) > 0:
        out.append(("cond_embed", (ch[0], int(lv["cond_dim"]), 1, 1)))
    return out


def unpack(lv: dict, flat: np.ndarray) -> dict:
    flat = np.asarray(flat, dtype=np.float32)
    shapes = param_shapes(lv)
    n = sum(int(np.prod(s)) for _, s in shapes)
    if flat.size != n:
        raise ValueError(f"weight vector has {flat.size} values, the network needs {n}")
    params, o = {}, 0
    for name, s in shapes:
        k = int(np.prod(s))
        params[name] = flat[o:o + k].astype(np.float64).reshape(s)
        o += k
    return params


# ---------------------------------------------------------------- layers

def conv(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Zero-padded stride-1 cross-correlation; x (B,C,H,W), w (Co,C,k,k)."""
    B, C, H, W = x.shape
    Co, Ci, kh, kw = w.shape
    assert Ci == C
    if kh == 1:
        y = np.einsum("bchw,oc->bohw", x, w[:, :, 0, 0], optimize=True)
        return y
    p = kh // 2
    xp = np.pad(x, ((0, 0), (0, 0), (p, p), (p, p)))
    out = np.empty((B, Co, H, W), dtype=np.float64)
    wm = w.reshape(Co, C * kh * kw).T
    for b in range(B):
        win = np.lib.stride_tricks.sliding_window_view(xp[b], (kh, kw), axis=(1, 2))
        cols = np.ascontiguousarray(win.transpose(1, 2, 0, 3, 4)).reshape(H * W, C * kh * kw)
        out[b] = (cols @ wm).T.reshape(Co, H, W)
    return out


def group_norm(x: np.ndarray, groups: int) -> np.ndarray:
    B, C, H, W = x.shape
    g = x.reshape(B, groups, -1)
    mean = g.mean(axis=2, keepdims=True)
    var = ((g - mean) ** 2).mean(axis=2, keepdims=True)
    return ((g - mean) / np.sqrt(var + GN_EPS)).reshape(B, C, H, W)


def silu(x: np.ndarray) -> np.ndarray:
    return x / (1.0 + np.exp(-x))


def avg_pool2(x: np.ndarray) -> np.ndarray:
    B, C, H, W = x.shape
    return x.reshape(B, C, H // 2, 2, W // 2, 2).mean(axis=(3, 5))


def up2(x: np.ndarray) -> np.ndarray:
    return x.repeat(2, axis=2).repeat(2, axis=3)


def resblock(x, p, name, groups):
    h = conv(silu(group_norm(x, groups)), p[name + ".conv1"])
    h = conv(silu(group_norm(h, groups)), p[name + ".conv2"])
    sk = p.get(name + ".skip")
    return h + (conv(x, sk) if sk is not None else x)


def attention(x, p, groups, heads):
    B, C, H, W = x.shape
    T = H * W
    d = C // heads
    h = group_norm(x, groups)
    qkv = conv(h, p["attn.qkv"]).reshape(B, 3, heads, d, T)
    q, k, v = qkv[:, 0], qkv[:, 1], qkv[:, 2]
    s = np.einsum("bhdt,bhds->bhts", q, k) / math.sqrt(d)
    s = s - s.max(axis=3, keepdims=True)
    e = np.exp(s)
    a = e / e.sum(axis=3, keepdims=True)
    o = np.einsum("bhts,bhds->bhdt", a, v).reshape(B, C, H, W)
    return x + conv(o, p["attn.proj"])


def cond_bias(p: dict, y: np.ndarray) -> np.ndarray:
    """Per-window bias E y (B, c0) of conditioning vectors y (B, D)."""
    return np.asarray(y, dtype=np.float64) @ p["cond_embed"][:, :, 0, 0].T


def forward(lv: dict, p: dict, x: np.ndarray, y=None) -> np.ndarray:
    """F(x) for a batch of windows x (B, in_ch, H, W) -> (B, out_ch, H, W);
    y (B, cond_dim): the windows' conditioning vectors (cond_dim > 0)."""
    td = int(lv.get("test_denoiser", 0))
    x = np.asarray(x, dtype=np.float64)
    if td:
        return test_denoiser(td, x)
    L = int(lv["levels"])
    G = int(lv["gn_groups"])
    h = conv(x, p["in_conv"])
    if y is not None:
        h = h + cond_bias(p, y)[:, :, None, None]
    skips = []
    for l in range(L):
        h = resblock(h, p, f"enc{l}", G)
        skips.append(h)
        if l < L - 1:
            h = avg_pool2(h)
    if int(lv.get("attn_at_bottom", 0)):
        h = attention(h, p, G, int(lv["attn_heads"]))
    h = resblock(h, p, "mid", G)
    for l in range(L - 2, -1, -1):
        h = np.concatenate([up2(h), skips[l]], axis=1)
        h = resblock(h, p, f"dec{l}", G)
    return conv(silu(group_norm(h, G)), p["out_conv"])


def test_denoiser(kind: int, x: np.ndarray) -> np.ndarray:
    B, C, H, W = x.shape
    if kind == 1:
        return np.full((B, 1, H, W), 0.5)
    s = x.sum(axis=1, keepdims=True)
    if kind == 2:
        return s
    if kind == 3:
        u = np.arange(H, dtype=np.float64)[:, None] / H
        v = np.arange(W, dtype=np.float64)[None, :] / W
        return s + (u - 2.0 * v)[None, None]
    raise ValueError(f"unknown test denoiser {kind}")


def flops_per_window(lv: dict) -> float:
    """Multiply-add FLOPs (2 per MAC) of the convolutions and attention
    matmuls of one window forward."""
    H = int(lv["window"])
    L = int(lv["levels"])
    ch = [int(c) for c in lv["channels"]]
    f = 0.0

    def c3(cin, cout, s):
        return 2.0 * 9 * cin * cout * s * s

    def rbf(cin, cout, s):
        v = c3(cin, cout, s) + c3(cout, cout, s)
        if cin != cout:
            v += 2.0 * cin * cout * s * s
        return v

    s = H
    f += c3(int(lv["in_ch"]), ch[0], s)
    prev = ch[0]
    for l in range(L):
        f += rbf(prev, ch[l], s)
        prev = ch[l]
        if l < L - 1:
            s //= 2
    if int(lv.get("attn_at_bottom", 0)):
        T = s * s
        C = prev
        f += 2.0 * T * C * 3 * C + 2.0 * T * C * C + 2.0 * 2.0 * T * T * C
    f += rbf(prev, prev, s)
    for l in range(L - 2, -1, -1):
        s *= 2
        f += rbf(prev + ch[l], ch[l], s)
        prev = ch[l]
    f += c3(prev, int(lv["out_ch"]), s)
    return f
