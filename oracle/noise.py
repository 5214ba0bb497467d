"""Seed function G(s, p): coordinate-keyed standard-normal noise (oracle).

Test infrastructure (see the package header).

The paper only requires that a seed deterministically fixes the initial noise
J_T(p) = G(s, p) (App. B, "Seeds and initial noise") and that re-noising be a
deterministic function of the seed (Sec. 3.5, seed consistency).  The reading
used here defines N(seed, level, step, x, y) bit for bit in IEEE-754 binary32:

1. Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
   easy as 1, 2, 3", SC'11): key = (seed mod 2^32, seed >> 32), counter =
   (x mod 2^32, y mod 2^32, step, level).  Only output words 0 and 1 are used.
2. u1 = ((o0 >> 8) + 1) * 2^-24 in (0, 1],  u2 = (o1 >> 8) * 2^-24 in [0, 1).
3. Box-Muller: z = sqrt(-2 ln u1) * cos(2 pi u2).

ln and cos are evaluated by polynomials written here from their series,
with every product and sum rounded separately to binary32 (no fused
multiply-add), so an independent implementation that follows the same
steps reproduces each value exactly:

* ln u: u = m 2^e with m in [1, 2), moved to [sqrt(2)/2, sqrt(2)] when its
  mantissa exceeds that of binary32 sqrt(2) (0x3FB504F3).  With z = (m-1)/(m+1)
  and w = z*z, ln m = 2z (1 + w/3 + w^2/5 + w^3/7 + w^4/9 + w^5/11) (the atanh
  series), evaluated as p = ((((c11 w + c9) w + c7) w + c5) w + c3) w, t = 2z,
  ln m = t + t*p with c_k = fl(1/k).  Then ln u = e*LN2_HI + (e*LN2_LO + ln m)
  (Cody-Waite split; LN2_HI = 22713/32768 holds 15 significant bits).
* cos 2 pi t, t = k 2^-24: quadrant q = (k + 2^21) >> 22, remainder
  r = (k - q 2^22) 2^-24 in [-1/8, 1/8), theta = r * fl(2 pi), x = theta^2;
  C = 1 + x(-1/2 + x(1/24 + x(-1/720 + x(1/40320 + x(-1/3628800
  + x/479001600))))),  S = theta + theta*x*(-1/6 + x(1/120 + x(-1/5040
  + x(1/362880 - x/39916800)))), each coefficient fl(+-1/n); the result is
  C, -S, -C, S for q mod 4 = 0, 1, 2, 3.

Pins (tests/test_oracle_noise.py): Philox known-answer vectors, the
polynomials against math.log / math.cos over their whole 2^24-point domains,
moments and a Kolmogorov-Smirnov test of the normals.
"""
from __future__ import annotations

import math

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 arrays (broadcast); returns 4 arrays."""
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    k0 = np.asarray(k0, dtype=np.uint32)
    k1 = np.asarray(k1, dtype=np.uint32)
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (a.copy() for a in (c0, c1, c2, c3))
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd > 0:
                k0 = (k0 + _W0).astype(np.uint32)
                k1 = (k1 + _W1).astype(np.uint32)
            p0 = _M0 * c0.astype(np.uint64)
            p1 = _M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            n0 = hi1 ^ c1 ^ k0
            n2 = hi0 ^ c3 ^ k1
            c0, c1, c2, c3 = n0, lo1, n2, lo0
    return c0, c1, c2, c3


_F = np.float32


def _c(n: int) -> np.float32:
    """fl(1/n) in binary32 (correctly rounded division of exact values)."""
    return np.divide(_F(1.0), _F(n), dtype=np.float32)


LN2_HI = _F(22713.0 / 32768.0)
LN2_LO = _F(math.log(2.0) - 22713.0 / 32768.0)
TWO_PI = _F(2.0 * math.pi)


def ln_f32(u: np.ndarray) -> np.ndarray:
    """Natural log of binary32 u > 0 (normal numbers), see the module header."""
    u = np.asarray(u, dtype=np.float32)
    bits = u.view(np.uint32)
    e = (bits >> np.uint32(23)).astype(np.int32) - 127
    mb = bits & np.uint32(0x7FFFFF)
    big = mb > np.uint32(0x3504F3)
    m = np.where(big, mb | np.uint32(0x3F000000), mb | np.uint32(0x3F800000)).astype(np.uint32).view(np.float32)
    e = np.where(big, e + 1, e)
    one = _F(1.0)
    f = m - one
    z = np.divide(f, m + one, dtype=np.float32)
    w = z * z
    p = _c(11) * w
    p = (p + _c(9)) * w
    p = (p + _c(7)) * w
    p = (p + _c(5)) * w
    p = (p + _c(3)) * w
    t = _F(2.0) * z
    lnm = t + t * p
    ef = e.astype(np.float32)
    r = ef * LN2_LO + lnm
    return (ef * LN2_HI + r).astype(np.float32)


def cos2pi_f32(k: np.ndarray) -> np.ndarray:
    """cos(2 pi k 2^-24) for integer k in [0, 2^24), see the module header."""
    k = np.asarray(k, dtype=np.int64)
    q = (k + (1 << 21)) >> 22
    rk = k - (q << 22)
    r = rk.astype(np.float32) * _F(2.0 ** -24)
    th = r * TWO_PI
    x = th * th
    cpoly = _c(479001600) * x + (-_c(3628800))
    cpoly = cpoly * x + _c(40320)
    cpoly = cpoly * x + (-_c(720))
    cpoly = cpoly * x + _c(24)
    cpoly = cpoly * x + _F(-0.5)
    C = _F(1.0) + x * cpoly
    spoly = -_c(39916800) * x + _c(362880)
    spoly = spoly * x + (-_c(5040))
    spoly = spoly * x + _c(120)
    spoly = spoly * x + (-_c(6))
    S = th + (th * x) * spoly
    n = (q & 3)
    out = np.where(n == 0, C, np.where(n == 1, -S, np.where(n == 2, -C, S)))
    return out.astype(np.float32)


def normal(seed: int, level: int, step: int, x, y) -> np.ndarray:
    """N(seed, level, step, x, y) as binary32; x, y int64 arrays (broadcast)."""
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    x, y = np.broadcast_arrays(x, y)
    cx = (x & 0xFFFFFFFF).astype(np.uint32)
    cy = (y & 0xFFFFFFFF).astype(np.uint32)
    seed = int(seed) & ((1 << 64) - 1)
    k0 = np.uint32(seed & 0xFFFFFFFF)
    k1 = np.uint32(seed >> 32)
    o0, o1, _, _ = philox4x32_10(cx, cy, np.uint32(step & 0xFFFFFFFF),
                                 np.uint32(level & 0xFFFFFFFF), k0, k1)
    a = (o0 >> np.uint32(8)).astype(np.int64) + 1
    b = (o1 >> np.uint32(8)).astype(np.int64)
    u1 = a.astype(np.float32) * _F(2.0 ** -24)
    l = ln_f32(u1)
    s = np.sqrt(_F(-2.0) * l, dtype=np.float32)
    c = cos2pi_f32(b)
    return (s * c).astype(np.float32)


def normal_region(seed: int, level: int, step: int, x0: int, y0: int, w: int, h: int) -> np.ndarray:
    """N over the region [y0, y0+h) x [x0, x0+w) as an (h, w) binary32 array."""
    ys = np.arange(y0, y0 + h, dtype=np.int64)[:, None]
    xs = np.arange(x0, x0 + w, dtype=np.int64)[None, :]
    return normal(seed, level, step, xs, ys)
