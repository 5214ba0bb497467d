"""Pins of the oracle's seed function G (noise), independent of the oracle itself."""
import math

import numpy as np
import pytest

from oracle import noise as N


# Known-answer vectors of Philox4x32-10 published with the algorithm
# (Salmon et al., SC'11, Random123 distribution): (counter, key) -> output.
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,out", KAT)
def test_philox_known_answers(ctr, key, out):
    r = N.philox4x32_10(*ctr, np.uint32(key[0]), np.uint32(key[1]))
    assert tuple(int(v) for v in r) == out


def test_ln_f32_whole_domain():
    # every u1 = k 2^-24 the noise can produce
    k = np.arange(1, 2 ** 24 + 1, dtype=np.int64)
    u = k.astype(np.float32) * np.float32(2.0 ** -24)
    got = N.ln_f32(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    ulp = np.spacing(np.abs(ref[:-1]).astype(np.float32)).astype(np.float64)
    assert got[-1] == 0.0
    assert np.max(np.abs(got[:-1] - ref[:-1]) / ulp) <= 2.0


def test_cos2pi_f32_whole_domain():
    k = np.arange(0, 2 ** 24, dtype=np.int64)
    got = N.cos2pi_f32(k).astype(np.float64)
    ref = np.cos(2.0 * np.pi * k / 2.0 ** 24)
    assert np.max(np.abs(got - ref)) <= 2.0 * 2.0 ** -24
    # exact at the quadrant points
    assert got[0] == 1.0 and got[1 << 22] == 0.0 and got[1 << 23] == -1.0


def test_normal_statistics():
    from scipy import stats
    n = 1 << 21
    x = np.arange(n, dtype=np.int64) % 4093 - 2000
    y = np.arange(n, dtype=np.int64) // 4093 - 100
    z = N.normal(12345, 1, 3, x, y).astype(np.float64)
    se = 1.0 / math.sqrt(n)
    assert abs(z.mean()) < 5 * se
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0) * se
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # third and fourth moments of a standard normal: 0 and 3
    assert abs((z ** 3).mean()) < 5 * math.sqrt(15.0) * se
    assert abs((z ** 4).mean() - 3.0) < 5 * math.sqrt(96.0) * se


def test_normal_counter_layout():
    # the counter is (x mod 2^32, y mod 2^32, step, level), key (seed lo, seed hi)
    seed = 0x0123456789ABCDEF
    z = N.normal(seed, 2, 5, np.array([-1, 7]), np.array([3, -2]))
    o0, o1, _, _ = N.philox4x32_10(np.array([0xFFFFFFFF, 7], np.uint32), np.array([3, 0xFFFFFFFE], np.uint32),
                                   5, 2, np.uint32(0x89ABCDEF), np.uint32(0x01234567))
    u1 = ((o0 >> np.uint32(8)).astype(np.float64) + 1) * 2.0 ** -24
    u2 = (o1 >> np.uint32(8)).astype(np.float64) * 2.0 ** -24
    ref = np.sqrt(-2 * np.log(u1)) * np.cos(2 * np.pi * u2)
    assert np.allclose(z, ref, rtol=1e-5, atol=1e-6)


def test_normal_decorrelated_across_step_level_seed():
    x = np.arange(200000) % 1000
    y = np.arange(200000) // 1000
    a = N.normal(0, 0, 0, x, y).astype(np.float64)
    for other in (N.normal(0, 0, 1, x, y), N.normal(0, 1, 0, x, y), N.normal(1, 0, 0, x, y)):
        c = np.corrcoef(a, other.astype(np.float64))[0, 1]
        assert abs(c) < 5 / math.sqrt(len(a))


def test_normal_region_matches_pointwise():
    r = N.normal_region(7, 0, 2, -5, 3, 4, 6)
    assert r.shape == (6, 4)
    assert r[2, 1] == N.normal(7, 0, 2, -4, 5)
