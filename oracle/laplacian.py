"""Signed square root and the Laplacian elevation encoding (oracle), FP64.

Test infrastructure (see the package header).

* Signed square root (Sec. 5.1, App. H): f(z) = sign(z) sqrt|z|, undone by
  f^-1(x) = sign(x) x^2.
* Laplacian encoding (Sec. 5.2): the low band is the image downsampled by the
  factor (8) and blurred (Gaussian, sigma = 5 low-resolution pixels); the
  residual is the image minus the upsampled low band.
* Laplacian denoising decode (Sec. 5.2): decode the generated pair (L, H)
  into a provisional image P = up(L) + H, re-extract the low band
  L^ = blur(down(P)), and synthesise L^ + H, i.e. v = up(L^) + H.  The
  alternative reading up(L^) + H^ with H^ = P - up(L^) would return P
  unchanged and is rejected.

Readings where the paper is silent: down = mean over the aligned factor x
factor block [f X, f X + f); up = bilinear with half-pixel centres,
u = (x + 1/2)/f - 1/2, whose weights are multiples of 1/(2f); blur taps
exp(-k^2 / (2 sigma^2)), |k| <= radius (15), normalised to sum 1; values are
denormalised before decoding as l = low_mu + low_scale L and h = res_scale H
(signed-sqrt units).  Decoding is defined pointwise on the infinite plane,
so a query reads L and H on a halo around itself (radius + 2 low-res pixels,
i.e. (radius + 1) f + f fine pixels).

Pins: f^-1(f(z)) = z; decode(encode(m)) = m; re-extraction is a fixed point
(L^ = L) when H is the exact residual; the gain of the re-extraction on
low-band noise equals its closed-form impulse response
(tests/test_oracle_laplacian.py).
"""
from __future__ import annotations

import math

import numpy as np


def signed_sqrt(z):
    z = np.asarray(z, dtype=np.float64)
    return np.sign(z) * np.sqrt(np.abs(z))


def signed_square(x):
    x = np.asarray(x, dtype=np.float64)
    return np.sign(x) * x * x


def blur_taps(sigma: float, radius: int) -> np.ndarray:
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    g = np.exp(-k * k / (2.0 * sigma * sigma))
    return g / g.sum()


def _up_index(c0: int, n: int, f: int):
    """For fine coordinates c0..c0+n-1: lower coarse index and weight of the
    upper neighbour under half-pixel-centred bilinear upsampling by f."""
    c = np.arange(c0, c0 + n, dtype=np.int64)
    num = 2 * c + 1 - f
    lo = num // (2 * f)
    a = (num - lo * 2 * f) / (2.0 * f)
    return lo, a


def up_bilinear(g: np.ndarray, gy0: int, gx0: int, y0: int, x0: int, h: int, w: int, f: int):
    """Bilinear upsampling by f of the coarse array g (origin gy0, gx0) over
    the fine rect (y0, x0, h, w)."""
    ly, ay = _up_index(y0, h, f)
    lx, ax = _up_index(x0, w, f)
    ry = ly - gy0
    rx = lx - gx0
    assert ry.min() >= 0 and ry.max() + 1 < g.shape[0], "coarse rows missing"
    assert rx.min() >= 0 and rx.max() + 1 < g.shape[1], "coarse cols missing"
    t = (1.0 - ay)[:, None] * g[ry] + ay[:, None] * g[ry + 1]
    return (1.0 - ax)[None, :] * t[:, rx] + ax[None, :] * t[:, rx + 1]


def up_range(c0: int, n: int, f: int):
    """Coarse index range [a, b] that bilinear upsampling of fine [c0, c0+n) reads."""
    a = (2 * c0 + 1 - f) // (2 * f)
    b = (2 * (c0 + n - 1) + 1 - f) // (2 * f) + 1
    return a, b


def down_mean(P: np.ndarray, f: int) -> np.ndarray:
    h, w = P.shape
    return P.reshape(h // f, f, w // f, f).mean(axis=(1, 3))


def blur2d_valid(D: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Separable blur keeping only outputs whose full stencil lies inside D."""
    R = (len(g) - 1) // 2
    h, w = D.shape
    t = np.zeros((h - 2 * R, w))
    for k in range(2 * R + 1):
        t += g[k] * D[k:k + h - 2 * R, :]
    out = np.zeros((h - 2 * R, w - 2 * R))
    for k in range(2 * R + 1):
        out += g[k] * t[:, k:k + w - 2 * R]
    return out


def decode_rects(y0, x0, h, w, *, factor=8, radius=15):
    """The rects (y0, x0, h, w) of L (coarse grid) and of H (fine grid) that
    the decode of the fine rect reads: the coarse range of L^ read by the
    final upsampling, grown by the blur radius, is D = down(P) over its
    aligned fine blocks, and P there reads L through one more upsampling."""
    f = int(factor)
    R = int(radius)
    qy0, qy1 = up_range(y0, h, f)
    qx0, qx1 = up_range(x0, w, f)
    dy0, dy1 = qy0 - R, qy1 + R
    dx0, dx1 = qx0 - R, qx1 + R
    py0, px0 = f * dy0, f * dx0
    ph, pw = f * (dy1 - dy0 + 1), f * (dx1 - dx0 + 1)
    ly0, ly1 = up_range(py0, ph, f)
    lx0, lx1 = up_range(px0, pw, f)
    return (ly0, lx0, ly1 - ly0 + 1, lx1 - lx0 + 1), (py0, px0, ph, pw)


def decode_signed(Lfun, Hfun, y0, x0, h, w, *, factor=8, blur_sigma=5.0, radius=15,
                  low_mu=0.0, low_scale=50.0, res_scale=1.5):
    """v = up(L^) + H over the fine rect (signed-sqrt units).

    Lfun(cy0, cx0, ch, cw): normalised low band on the coarse grid.
    Hfun(y0, x0, h, w): normalised residual on the fine grid."""
    f = int(factor)
    R = int(radius)
    g = blur_taps(blur_sigma, R)
    (ly0, lx0, lh, lw), (py0, px0, ph, pw) = decode_rects(y0, x0, h, w, factor=f, radius=R)
    # coarse rows/cols of L^ the final upsampling reads
    qy0, qy1 = up_range(y0, h, f)
    qx0, qx1 = up_range(x0, w, f)
    l = low_mu + low_scale * np.asarray(Lfun(ly0, lx0, lh, lw), dtype=np.float64)
    hP = res_scale * np.asarray(Hfun(py0, px0, ph, pw), dtype=np.float64)
    P = up_bilinear(l, ly0, lx0, py0, px0, ph, pw, f) + hP
    D = down_mean(P, f)
    Lhat = blur2d_valid(D, g)          # rows qy0..qy1, cols qx0..qx1
    v = up_bilinear(Lhat, qy0, qx0, y0, x0, h, w, f)
    v = v + hP[y0 - py0:y0 - py0 + h, x0 - px0:x0 - px0 + w]
    return v


def decode_metres(Lfun, Hfun, y0, x0, h, w, **kw):
    return signed_square(decode_signed(Lfun, Hfun, y0, x0, h, w, **kw))


def encode_funcs(field, *, factor=8, blur_sigma=5.0, radius=15,
                 low_mu=0.0, low_scale=50.0, res_scale=1.5):
    """Laplacian encoding of a signed-sqrt field given as field(y0, x0, h, w)
    on the fine grid.  Returns (Lfun, Hfun), the normalised bands as
    functions of a rect, for round-trip tests."""
    f = int(factor)
    R = int(radius)
    g = blur_taps(blur_sigma, R)

    def low(cy0, cx0, ch, cw):
        D = down_mean(field(f * (cy0 - R), f * (cx0 - R), f * (ch + 2 * R), f * (cw + 2 * R)), f)
        return blur2d_valid(D, g)

    def Lfun(cy0, cx0, ch, cw):
        return (low(cy0, cx0, ch, cw) - low_mu) / low_scale

    def Hfun(y0, x0, h, w):
        a0, a1 = up_range(y0, h, f)
        b0, b1 = up_range(x0, w, f)
        lo = low(a0, b0, a1 - a0 + 1, b1 - b0 + 1)
        return (field(y0, x0, h, w) - up_bilinear(lo, a0, b0, y0, x0, h, w, f)) / res_scale

    return Lfun, Hfun


def periodic_field(arr: np.ndarray):
    """field(y0, x0, h, w) reading a periodic 2-D array."""
    arr = np.asarray(arr, dtype=np.float64)
    Py, Px = arr.shape

    def field(y0, x0, h, w):
        ys = np.arange(y0, y0 + h) % Py
        xs = np.arange(x0, x0 + w) % Px
        return arr[np.ix_(ys, xs)]

    return field


def periodic_lowband(arr: np.ndarray):
    """Lfun reading a periodic coarse array of *signed-sqrt* low-band values
    (normalisation is applied by the caller through low_mu / low_scale = 0 / 1)."""
    return periodic_field(arr)
