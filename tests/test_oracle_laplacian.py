"""Pins of the oracle's signed square root and Laplacian encode / decode."""
import numpy as np
import pytest

from oracle import laplacian as L


def test_signed_sqrt_pair():
    z = np.array([-11000.0, -3.5, -1e-9, 0.0, 2e-7, 1.0, 8848.0])
    assert np.allclose(L.signed_square(L.signed_sqrt(z)), z, rtol=1e-15, atol=0)
    assert L.signed_sqrt(-4.0) == -2.0 and L.signed_square(-3.0) == -9.0


def test_blur_taps():
    g = L.blur_taps(5.0, 15)
    assert len(g) == 31 and g.sum() == pytest.approx(1.0, abs=1e-15)
    assert g[15] / g[16] == pytest.approx(np.exp(1.0 / 50.0), rel=1e-14)
    assert np.allclose(g, g[::-1])


def test_up_weights_are_half_pixel_centred():
    # fine pixel x = 8 X + r reads coarse X-1, X (r < 4) or X, X+1 (r >= 4)
    lo, a = L._up_index(0, 8, 8)
    assert list(lo) == [-1, -1, -1, -1, 0, 0, 0, 0]
    assert list(a * 16) == [9, 11, 13, 15, 1, 3, 5, 7]
    # upsampling a linear ramp reproduces the ramp at the coarse pixel centres
    g = np.arange(10, dtype=np.float64)[:, None] * np.ones((1, 10))
    u = L.up_bilinear(g, 0, 0, 8, 8, 64, 8, 8)
    assert np.allclose(u[:, 0], (np.arange(8, 72) + 0.5) / 8 - 0.5)


def _periodic_terrain(n=64, seed=0):
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((n, n))
    # smooth-ish field in signed-sqrt units spanning +-100 (about +-10 km)
    F = np.fft.fft2(f)
    ky = np.fft.fftfreq(n)[:, None]
    kx = np.fft.fftfreq(n)[None, :]
    F *= 1.0 / (1.0 + 40.0 * np.sqrt(kx * kx + ky * ky))
    x = np.real(np.fft.ifft2(F))
    return 100.0 * x / np.abs(x).max()


@pytest.mark.parametrize("rect", [(0, 0, 40, 40), (-77, 301, 23, 57), (5, -9, 1, 1)])
def test_encode_decode_round_trip(rect):
    field = L.periodic_field(_periodic_terrain(512))
    Lf, Hf = L.encode_funcs(field)
    got = L.decode_metres(Lf, Hf, *rect)
    ref = L.signed_square(field(*rect))
    assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_reextraction_is_a_fixed_point():
    # with H the exact residual, blur(down(up(L) + H)) returns L itself
    field = L.periodic_field(_periodic_terrain(512, 1))
    Lf, Hf = L.encode_funcs(field, low_mu=3.0, low_scale=20.0, res_scale=2.0)
    v = L.decode_signed(Lf, Hf, 16, 24, 32, 48, low_mu=3.0, low_scale=20.0, res_scale=2.0)
    assert np.max(np.abs(v - field(16, 24, 32, 48))) < 1e-10


def test_lowband_noise_gain_matches_impulse_response():
    # An impulse e on the low band at coarse (Y, X) changes the decode by
    # low_scale * up(blur(down(up(e)))).  The 1-D response of down(up(.)) by
    # f = 8 with half-pixel bilinear weights is [1/8, 3/4, 1/8]: block X sees
    # its own value with weight 1 - 2 * (sum_{r<4} (7-2r)/16)/8 = 3/4 and each
    # neighbour with (1 + 3 + 5 + 7)/16/8 = 1/8.
    field = L.periodic_field(_periodic_terrain(512, 2))
    Lf, Hf = L.encode_funcs(field)
    Y, X = 3, 4

    def Lpert(cy0, cx0, ch, cw):
        a = Lf(cy0, cx0, ch, cw).copy()
        if cy0 <= Y < cy0 + ch and cx0 <= X < cx0 + cw:
            a[Y - cy0, X - cx0] += 1.0
        return a

    rect = (0, 0, 64, 64)
    d = L.decode_signed(Lpert, Hf, *rect) - L.decode_signed(Lf, Hf, *rect)
    k = np.array([1 / 8, 3 / 4, 1 / 8])
    g = L.blur_taps(5.0, 15)
    r1 = np.convolve(g, k)                      # 33 taps centred at index 16
    # coarse response on rows/cols -1..40 (fine 0..63 reads coarse -1..8)
    resp = np.zeros((42, 42))
    for a in range(-1, 41):
        for b in range(-1, 41):
            ia, ib = a - Y + 16, b - X + 16
            if 0 <= ia < 33 and 0 <= ib < 33:
                resp[a + 1, b + 1] = r1[ia] * r1[ib]
    ref = 50.0 * L.up_bilinear(resp, -1, -1, 0, 0, 64, 64, 8)
    assert np.max(np.abs(d - ref)) < 1e-12
    # the re-extraction attenuates white low-band noise: sum of squared taps < 1
    assert (r1 ** 2).sum() ** 2 < 0.02


def test_periodic_field_wraps_by_brute_force():
    # periodic reads at negative and beyond-period coordinates equal the
    # array entry at (y mod P, x mod P), element by element
    rng = np.random.default_rng(5)
    arr = rng.standard_normal((7, 5))
    f = L.periodic_field(arr)
    y0, x0, h, w = -9, 3, 20, 13
    got = f(y0, x0, h, w)
    for i in range(h):
        for j in range(w):
            assert got[i, j] == arr[(y0 + i) % 7, (x0 + j) % 5]


def test_world_metres_reads_a_given_low_band():
    # a single-level Laplacian stack with a given periodic low band decodes
    # exactly that band with the level's residual (the low band is read here
    # by explicit loops, independently of periodic_field)
    import synth
    from oracle import sampler as OS
    rng = np.random.default_rng(6)
    fx = (rng.standard_normal((16, 16)) * 30.0).astype(np.float32)
    st = synth.config4_stack(fx, steps=2, test_denoiser=2)
    W = OS.World(0, st, [None])

    def lfun(cy0, cx0, ch, cw):
        out = np.empty((ch, cw))
        for i in range(ch):
            for j in range(cw):
                out[i, j] = fx[(cy0 + i) % 16, (cx0 + j) % 16]
        return out

    rect = (-20, 100, 24, 30)
    got = W.metres(*rect)
    ref = L.decode_metres(lfun, W.levels[0].final, *rect, factor=8, blur_sigma=5.0, radius=15,
                          low_mu=0.0, low_scale=1.0, res_scale=1.5)
    assert np.array_equal(got, ref)
