"""InfiniteDiffusion on Z^3 (oracle): windowed sampling of unbounded voxel
volumes, FP64.

Test infrastructure (see the package header).

The method is defined on S = Z^d (Sec. 3.2; Alg. 3 computes kappa per
dimension; the conclusion names voxel volumes).  This module restates the
2-D oracle for d = 3 with the same readings:

* windows (i, j, l) cover [i s, i s + H) x [j s, j s + H) x [l s, l s + H)
  (z, y, x order); kappa per axis as oracle.kappa.kappa_1d;
* weights W(u, v, w) = w1(u) w1(v) w1(w) with the separable linear w1 of
  Sec. 6 (oracle.schedule.weight_1d), blending by Eq. 2;
* noise N3(seed, level, step, x, y, z): the seed function of App. B on Z^3,
  Philox4x32-10 with counter (x mod 2^32, y mod 2^32, z mod 2^32,
  2^31 + level 2^16 + step) -- the top bit keeps it apart from the 2-D
  counter (x, y, step, level) -- and the 2-D module's Box-Muller in binary32;
* one blended step per round, EDM preconditioning and sigma schedule as in
  2-D (oracle.schedule);
* the denoiser: a small 3-D network F(x) = conv3(silu(gn(conv3(x)))) with C
  hidden channels, 3 x 3 x 3 zero-padded convolutions per window, GroupNorm
  of G groups (population variance, eps 1e-5), no biases (the synthetic
  stand-in of a voxel model; the paper trains none), or a closed-form test
  denoiser (1 constant 0.5, 2 identity, 3 identity + u/H - 2 v/H + 3 w/H in
  window-local z, y, x).

Routes: ``VolumeLevel`` is Alg. 1 (lazy, per-window contributions, every
window evaluated once); ``eager_volume`` is Eq. 1 on a canvas holding the
whole cone.  Pins: the two routes agree; closed forms of the test
denoisers; the network against torch.nn.functional.conv3d / group_norm;
window counts sum_k (n + 2k + 1)^3 (tests/test_oracle_volume.py).
"""
from __future__ import annotations

import math

import numpy as np

from . import kappa as K_
from . import noise as N_
from . import schedule as S_


def normal3(seed: int, level: int, step: int, x, y, z) -> np.ndarray:
    """N3(seed, level, step, x, y, z) as binary32 (int64 arrays, broadcast)."""
    x, y, z = (np.asarray(a, dtype=np.int64) for a in (x, y, z))
    x, y, z = np.broadcast_arrays(x, y, z)
    c3 = np.uint32((1 << 31) + ((int(level) & 0x7FFF) << 16) + (int(step) & 0xFFFF))
    seed = int(seed) & ((1 << 64) - 1)
    o0, o1, _, _ = N_.philox4x32_10((x & 0xFFFFFFFF).astype(np.uint32), (y & 0xFFFFFFFF).astype(np.uint32),
                                    (z & 0xFFFFFFFF).astype(np.uint32), c3, np.uint32(seed & 0xFFFFFFFF),
                                    np.uint32(seed >> 32))
    a = (o0 >> np.uint32(8)).astype(np.int64) + 1
    b = (o1 >> np.uint32(8)).astype(np.int64)
    u1 = a.astype(np.float32) * np.float32(2.0 ** -24)
    s = np.sqrt(np.float32(-2.0) * N_.ln_f32(u1), dtype=np.float32)
    return (s * N_.cos2pi_f32(b)).astype(np.float32)


def normal3_box(seed, level, step, z0, y0, x0, d, h, w) -> np.ndarray:
    """N3 over [z0, z0+d) x [y0, y0+h) x [x0, x0+w) as a (d, h, w) array."""
    zs = np.arange(z0, z0 + d, dtype=np.int64)[:, None, None]
    ys = np.arange(y0, y0 + h, dtype=np.int64)[None, :, None]
    xs = np.arange(x0, x0 + w, dtype=np.int64)[None, None, :]
    return normal3(seed, level, step, xs, ys, zs)


# ---------------------------------------------------------------- network

def param_shapes(desc: dict):
    C = int(desc["channels"])
    return [("conv1", (C, 1, 3, 3, 3)), ("conv2", (1, C, 3, 3, 3))]


def unpack(desc: dict, flat) -> dict:
    flat = np.asarray(flat, dtype=np.float32)
    out, o = {}, 0
    for name, s in param_shapes(desc):
        k = int(np.prod(s))
        out[name] = flat[o:o + k].astype(np.float64).reshape(s)
        o += k
    if o != flat.size:
        raise ValueError("weight vector does not match the volume network")
    return out


def conv3(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Zero-padded 3x3x3 cross-correlation; x (B, C, D, H, W), w (Co, C, 3, 3, 3)."""
    B, C, D, H, W = x.shape
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1), (1, 1)))
    wm = w.reshape(w.shape[0], -1).T
    out = np.empty((B, w.shape[0], D, H, W))
    for b in range(B):
        win = np.lib.stride_tricks.sliding_window_view(xp[b], (3, 3, 3), axis=(1, 2, 3))
        cols = np.ascontiguousarray(win.transpose(1, 2, 3, 0, 4, 5, 6)).reshape(D * H * W, -1)
        out[b] = (cols @ wm).T.reshape(-1, D, H, W)
    return out


def group_norm(x: np.ndarray, groups: int) -> np.ndarray:
    B, C = x.shape[:2]
    g = x.reshape(B, groups, -1)
    m = g.mean(axis=2, keepdims=True)
    v = ((g - m) ** 2).mean(axis=2, keepdims=True)
    return ((g - m) / np.sqrt(v + 1e-5)).reshape(x.shape)


def forward(desc: dict, p, x: np.ndarray) -> np.ndarray:
    """F of windows x (B, 1, H, H, H) -> (B, 1, H, H, H)."""
    td = int(desc.get("test_denoiser", 0))
    x = np.asarray(x, dtype=np.float64)
    if td == 1:
        return np.full_like(x, 0.5)
    if td == 2:
        return x.copy()
    if td == 3:
        H = x.shape[-1]
        u = np.arange(H, dtype=np.float64) / H
        return x + (u[:, None, None] - 2.0 * u[None, :, None] + 3.0 * u[None, None, :])[None, None]
    h = conv3(x, p["conv1"])
    h = group_norm(h, int(desc["groups"]))
    h = h / (1.0 + np.exp(-h))
    return conv3(h, p["conv2"])


# ---------------------------------------------------------------- sampler

class _Common:
    def __init__(self, seed: int, desc: dict, weights=None, level: int = 0):
        self.seed, self.level, self.desc = int(seed), int(level), dict(desc)
        self.H, self.s, self.K = int(desc["window"]), int(desc["stride"]), int(desc["steps"])
        self.sig = S_.sigmas(self.K, desc["sigma_max"], desc["sigma_min"], desc["rho"])
        self.sd = float(desc["sigma_data"])
        w1 = S_.weight_1d(self.H, float(desc.get("blend_eps", 1e-3)))
        self.W = w1[:, None, None] * w1[None, :, None] * w1[None, None, :]
        self.params = unpack(desc, weights) if int(desc.get("test_denoiser", 0)) == 0 else None
        self.phi_calls = 0

    def noise(self, step, z0, y0, x0, d, h, w):
        return normal3_box(self.seed, self.level, step, z0, y0, x0, d, h, w).astype(np.float64)

    def rect(self, key):
        i, j, l = key
        return (i * self.s, j * self.s, l * self.s)

    def phi(self, k, xs, keys):
        """One sampler step of every window: D(x; sigma_k) + sigma_{k+1} N3."""
        c_skip, c_out, c_in = S_.edm_coeffs(self.sig[k], self.sd)
        xin = np.stack(xs)[:, None] * c_in
        F = np.concatenate([forward(self.desc, self.params, xin[b:b + 8]) for b in range(0, len(xs), 8)])[:, 0]
        self.phi_calls += len(xs)
        out = []
        for x, key, f in zip(xs, keys, F):
            dd = c_skip * x + c_out * f
            if k + 1 < self.K:
                dd = dd + self.sig[k + 1] * self.noise(k + 1, *self.rect(key), self.H, self.H, self.H)
            out.append(dd)
        return out


def kappa3(z0, y0, x0, d, h, w, H, s):
    """Windows (i, j, l) meeting the box, sorted (Alg. 3 per axis)."""
    rz = K_.kappa_1d(z0, z0 + d, H, s)
    ry = K_.kappa_1d(y0, y0 + h, H, s)
    rx = K_.kappa_1d(x0, x0 + w, H, s)
    if rz is None or ry is None or rx is None:
        return []
    return [(i, j, l) for i in range(rz[0], rz[1] + 1) for j in range(ry[0], ry[1] + 1)
            for l in range(rx[0], rx[1] + 1)]


class VolumeLevel(_Common):
    """Alg. 1 on Z^3: J_k of a box from the windows' contributions (each
    window evaluated once, kept per step)."""

    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.contrib = [dict() for _ in range(self.K + 1)]

    def J(self, k, z0, y0, x0, d, h, w):
        if k == 0:
            return self.sig[0] * self.noise(0, z0, y0, x0, d, h, w)
        win = kappa3(z0, y0, x0, d, h, w, self.H, self.s)
        store = self.contrib[k]
        todo = [key for key in win if key not in store]
        if todo:
            xs = [self.J(k - 1, *self.rect(key), self.H, self.H, self.H) for key in todo]
            for key, p in zip(todo, self.phi(k - 1, xs, todo)):
                store[key] = self.W * p
        A = np.zeros((d, h, w))
        B = np.zeros((d, h, w))
        for key in win:
            a0, b0, c0 = self.rect(key)
            za, zb = max(z0, a0), min(z0 + d, a0 + self.H)
            ya, yb = max(y0, b0), min(y0 + h, b0 + self.H)
            xa, xb = max(x0, c0), min(x0 + w, c0 + self.H)
            sl = (slice(za - z0, zb - z0), slice(ya - y0, yb - y0), slice(xa - x0, xb - x0))
            ws = (slice(za - a0, zb - a0), slice(ya - b0, yb - b0), slice(xa - c0, xb - c0))
            A[sl] += store[key][ws]
            B[sl] += self.W[ws]
        out = np.zeros((d, h, w))
        nz = B != 0
        out[nz] = A[nz] / B[nz]
        return out

    def final(self, z0, y0, x0, d, h, w):
        return self.J(self.K, z0, y0, x0, d, h, w)


def eager_volume(seed, desc, weights, z0, y0, x0, d, h, w, level=0):
    """Eq. 1 on a canvas holding the box's whole cone."""
    lv = _Common(seed, desc, weights, level)
    H, s, K = lv.H, lv.s, lv.K
    box = (z0, y0, x0, d, h, w)
    for _ in range(K):
        rz = K_.kappa_1d(box[0], box[0] + box[3], H, s)
        ry = K_.kappa_1d(box[1], box[1] + box[4], H, s)
        rx = K_.kappa_1d(box[2], box[2] + box[5], H, s)
        box = (rz[0] * s, ry[0] * s, rx[0] * s, (rz[1] - rz[0]) * s + H, (ry[1] - ry[0]) * s + H,
               (rx[1] - rx[0]) * s + H)
    cz, cy, cx, cd, ch, cw = box
    J = lv.sig[0] * lv.noise(0, cz, cy, cx, cd, ch, cw)
    keys = kappa3(cz, cy, cx, cd, ch, cw, H, s)
    keys = [k for k in keys if all(k[a] * s >= box[a] and k[a] * s + H <= box[a] + box[3 + a] for a in range(3))]
    for k in range(K):
        xs = []
        for key in keys:
            a0, b0, c0 = lv.rect(key)
            xs.append(J[a0 - cz:a0 - cz + H, b0 - cy:b0 - cy + H, c0 - cx:c0 - cx + H])
        phis = lv.phi(k, xs, keys)
        A = np.zeros(J.shape)
        B = np.zeros(J.shape)
        for key, p in zip(keys, phis):
            a0, b0, c0 = lv.rect(key)
            sl = (slice(a0 - cz, a0 - cz + H), slice(b0 - cy, b0 - cy + H), slice(c0 - cx, c0 - cx + H))
            A[sl] += lv.W * p
            B[sl] += lv.W
        J = np.zeros(J.shape)
        nz = B != 0
        J[nz] = A[nz] / B[nz]
    return J[z0 - cz:z0 - cz + d, y0 - cy:y0 - cy + h, x0 - cx:x0 - cx + w]
