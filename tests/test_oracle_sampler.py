"""Pins of the oracle sampler: closed forms, Lemma 3 (lazy == eager),
Thm 1 (order / cache independence), window accounting (Lemma 4)."""
import math

import numpy as np
import pytest

import synth
from oracle import kappa as K
from oracle import noise as N
from oracle import sampler as S
from oracle import schedule as Sc
from oracle import unet as U


def _weights(st, seed=0):
    return [synth.weights([s for _, s in U.param_shapes(lv)], seed, li) for li, lv in enumerate(st["level"])]


# ----------------------------------------------------------- schedule pieces

def test_sigma_schedule():
    s = Sc.sigmas(4, 80.0, 0.02, 7.0)
    assert s[0] == pytest.approx(80.0, rel=1e-15) and s[-1] == pytest.approx(0.02, rel=1e-12)
    assert np.all(np.diff(s) < 0)
    assert s[1] == pytest.approx(12.67583, rel=1e-5) and s[2] == pytest.approx(1.032751, rel=1e-5)
    s20 = Sc.sigmas(20, 80.0, 0.02, 7.0)
    assert s20[1] == pytest.approx(61.650, rel=1e-4) and s20[-2] == pytest.approx(0.04407, rel=1e-3)


def test_edm_identity():
    # c_skip + c_out^2 / sd^2 = 1 and c_in^2 (sigma^2 + sd^2) = 1
    for sig in [80.0, 1.0, 0.02]:
        cs, co, ci = Sc.edm_coeffs(sig, 0.5)
        assert cs + co * co / 0.25 == pytest.approx(1.0, abs=1e-14)
        assert ci * ci * (sig * sig + 0.25) == pytest.approx(1.0, abs=1e-14)


def test_weight_window_and_denominator():
    for s in (16, 64, 5):
        H = 2 * s
        w = Sc.weight_1d(H, 1e-3)
        assert w[0] == pytest.approx(1e-3) and w[-1] == pytest.approx(1e-3)
        assert np.all(w <= 1.0) and np.all(w > 0)
        # per-axis sum of the two windows covering a pixel is constant
        B1 = w[:s] + w[s:]
        assert np.allclose(B1, 2.0 - (1.0 - 1e-3) * s / (s - 0.5), rtol=1e-14)
    assert 2.0 - 0.999 * 16 / 15.5 == pytest.approx(0.9687742, abs=1e-7)


# ----------------------------------------------------------- closed forms

def _closed_form_pixelwise(lv, seed, level_index, y0, x0, h, w, F_of_J):
    """J_{k+1} = c_skip J_k + c_out Fbar_k + sigma_{k+1} N per pixel."""
    K_ = lv["steps"]
    sig = Sc.sigmas(K_, lv["sigma_max"], lv["sigma_min"], lv["rho"])
    J = sig[0] * N.normal_region(seed, level_index, 0, x0, y0, w, h).astype(np.float64)
    for k in range(K_):
        cs, co, ci = Sc.edm_coeffs(sig[k], lv["sigma_data"])
        J = cs * J + co * F_of_J(J, ci, k)
        if k + 1 < K_:
            J = J + sig[k + 1] * N.normal_region(seed, level_index, k + 1, x0, y0, w, h)
    return J


@pytest.mark.parametrize("td", [1, 2])
def test_constant_and_identity_denoisers_closed_form(td):
    st = synth.config1_stack(test_denoiser=td)
    lv = st["level"][0]
    world = S.World(3, st, None)
    got = world.model(-40, 17, 37, 29)
    F = (lambda J, ci, k: 0.5) if td == 1 else (lambda J, ci, k: ci * J)
    ref = _closed_form_pixelwise(lv, 3, 0, -40, 17, 37, 29, F)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_local_coordinate_denoiser_closed_form():
    # F = c_in J + u/H - 2 v/H: the blend adds sum_i W_i g_i / sum_i W_i with g
    # the window-local coordinate term, written out here per pixel.
    st = synth.config1_stack(test_denoiser=3)
    lv = st["level"][0]
    H, s = lv["window"], lv["stride"]
    world = S.World(5, st, None)
    y0, x0, h, w = -23, 40, 19, 21
    got = world.model(y0, x0, h, w)
    w1 = Sc.weight_1d(H, 1e-3)
    g = np.zeros((h, w))
    for a in range(h):
        Y = y0 + a
        for b in range(w):
            X = x0 + b
            num = den = 0.0
            for i in range(Y // s - 1, Y // s + 1):
                for j in range(X // s - 1, X // s + 1):
                    u, v = Y - i * s, X - j * s
                    ww = w1[u] * w1[v]
                    num += ww * (u / H - 2.0 * v / H)
                    den += ww
            g[a, b] = num / den
    ref = _closed_form_pixelwise(lv, 5, 0, y0, x0, h, w, lambda J, ci, k: ci * J + g)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


# ----------------------------------------------------------- lazy == eager

def test_lazy_equals_eager_config1_arch():
    st = synth.with_steps(synth.config1_stack(), 2)
    wts = _weights(st)
    lazy = S.World(0, st, wts).model(-5, 9, 20, 23)
    eager = S.eager_world_model(0, st, wts, -5, 9, 20, 23)
    assert np.max(np.abs(lazy - eager)) <= 1e-12 * np.max(np.abs(eager))


def test_lazy_equals_eager_two_level():
    st = synth.small_hier_stack(steps=2, window=16, stride=8, coarse_channels=(8, 8),
                                fine_channels=(8, 8))
    wts = _weights(st)
    lazy = S.World(1, st, wts).model(3, -20, 12, 10)
    eager = S.eager_world_model(1, st, wts, 3, -20, 12, 10)
    assert np.max(np.abs(lazy - eager)) <= 1e-12 * np.max(np.abs(eager))


def test_cone_eager_equals_dense_eager_term_for_term():
    # the eager form that evaluates only the windows covering each round's
    # needed region sums, at every needed pixel, the same terms in the same
    # order as the dense form over the whole canvas: equal bit for bit, with
    # fewer evaluations
    cases = [
        (synth.with_steps(synth.config1_stack(), 3), (-5, 9, 20, 23)),
        (synth.small_hier_stack(steps=2, window=16, stride=8, coarse_channels=(8, 8), fine_channels=(8, 8)),
         (3, -20, 12, 10)),
        (synth.with_steps(synth.config1_stack(test_denoiser=3), 4), (-40, 7, 33, 18)),
    ]
    for st, (y0, x0, h, w) in cases:
        wts = _weights(st) if not st["level"][0].get("test_denoiser") else None
        a = S.eager_world_model(2, st, wts, y0, x0, h, w)
        b = S.eager_world_model(2, st, wts, y0, x0, h, w, dense=True)
        assert np.array_equal(a, b)
    lv = synth.with_steps(synth.config1_stack(test_denoiser=3), 4)["level"][0]
    c, d = S.EagerLevel(0, lv, 0), S.EagerLevel(0, lv, 0)
    assert np.array_equal(c.run(0, 0, 16, 16), d.run(0, 0, 16, 16, dense=True))
    assert c.phi_calls < d.phi_calls


# ----------------------------------------------------------- Thm 1, Lemma 4

def test_order_and_cache_independence():
    st = synth.with_steps(synth.config1_stack(), 3)
    wts = _weights(st)
    r1, r2 = (0, 0, 40, 40), (20, 24, 40, 30)
    a = S.World(0, st, wts)
    a1, a2 = a.model(*r1), a.model(*r2)
    b = S.World(0, st, wts)
    b2, b1 = b.model(*r2), b.model(*r1)
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)
    # overlap agreement
    assert np.array_equal(a1[20:40, 24:40], a2[0:20, 0:16])
    for cap in (0, 1, 5):
        c = S.World(0, st, wts, capacity=cap)
        c.model(*r2)
        assert np.array_equal(c.model(*r1), a1)


def test_phi_call_accounting():
    st = synth.config1_stack(test_denoiser=1)
    world = S.World(0, st, None)
    world.model(0, 0, 64, 64)
    lvl = world.levels[0]
    assert lvl.phi_calls == 276
    # a repeated query is served from the contributions: no new Phi calls
    world.model(0, 0, 64, 64)
    assert lvl.phi_calls == 276
    # a neighbouring 64x64 query reuses overlapping windows
    world.model(0, 64, 64, 64)
    assert lvl.phi_calls < 2 * 276


def test_division_by_zero_is_zero():
    # stride > window leaves uncovered pixels: B = 0 there and J is defined as 0
    lv = synth.level(window=4, stride=6, steps=1, test_denoiser=1)
    world = S.World(0, synth.stack([lv]), None)
    out = world.model(0, 0, 1, 12)[0]
    assert np.all(out[4:6] == 0.0) and np.all(out[0:4] != 0.0)


def test_conditioning_closed_form_two_level():
    # Identity denoisers (F = sum of input channels) on a two-level stack: the
    # coarse level follows the one-channel closed form, and every fine pixel
    # (x, y) follows J <- c_skip J + c_out (c_in J + L(floor(x/8), floor(y/8)))
    # + sigma N with L the coarse result, unscaled (Sec. 5.3 conditioning by
    # nearest-neighbour upsampling).
    st = synth.small_hier_stack(steps=3, window=16, stride=8, test_denoiser=2)
    world = S.World(4, st, None)
    y0, x0, h, w = -13, 21, 11, 19
    got = world.model(y0, x0, h, w)
    coarse_lv, fine_lv = st["level"]
    cy0, cx0 = y0 // 8, x0 // 8
    cy1, cx1 = (y0 + h - 1) // 8, (x0 + w - 1) // 8
    Lc = _closed_form_pixelwise(coarse_lv, 4, 0, cy0, cx0, cy1 - cy0 + 1, cx1 - cx0 + 1,
                                lambda J, ci, k: ci * J)
    ys = np.arange(y0, y0 + h) // 8 - cy0
    xs = np.arange(x0, x0 + w) // 8 - cx0
    cond = Lc[np.ix_(ys, xs)]
    ref = _closed_form_pixelwise(fine_lv, 4, 1, y0, x0, h, w, lambda J, ci, k: ci * J + cond)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


# ----------------------------------------------------------- eager world (stored-fixture route)

def test_eager_world_with_pool_equals_lazy_world():
    # EagerWorld (Eq. 1 over the cone of the decode's halo, F evaluated in
    # worker processes) against the lazy Alg. 1 world: model units and metres
    from oracle import parallel as P
    st = synth.small_hier_stack(steps=1, fine_channels=(8, 16), coarse_channels=(8, 8))
    wts = _weights(st)
    y0, x0, h, w = 5, -7, 12, 10
    pool = P.PoolForward(st, wts, 2)
    try:
        ew = S.EagerWorld(3, st, wts, y0, x0, h, w, metres=True, fmap=pool.fmap)
    finally:
        pool.close()
    lz = S.World(3, st, wts)
    m_e, m_l = ew.model(y0, x0, h, w), lz.model(y0, x0, h, w)
    v_e, v_l = ew.metres(y0, x0, h, w), lz.metres(y0, x0, h, w)
    assert np.max(np.abs(m_e - m_l)) <= 1e-12 * np.max(np.abs(m_l))
    assert np.max(np.abs(v_e - v_l)) <= 1e-12 * np.max(np.abs(v_l))
    # the pooled F equals the serial one up to BLAS summation order
    e2 = S.EagerWorld(3, st, wts, y0, x0, h, w)
    assert np.max(np.abs(e2.model(y0, x0, h, w) - m_e)) <= 1e-13 * np.max(np.abs(m_e))


# ----------------------------------------------------------- T variants (rounds)

def _rounds(st, rounds):
    st = synth.with_steps(st, sum(rounds))
    st["level"][0]["round_steps"] = tuple(rounds)
    return st


@pytest.mark.parametrize("td", [1, 2])
def test_rounds_equal_per_step_for_pixel_local_denoisers(td):
    # with F independent of the window (constant, or the pixel's own value),
    # every covering window follows the same pixel trajectory, so blending
    # only at round ends changes nothing
    base = synth.config1_stack(test_denoiser=td)
    a = S.World(2, _rounds(base, (1, 1, 1, 1)), None).model(-9, 30, 21, 18)
    for rs in ((2, 2), (4,), (1, 3)):
        b = S.World(2, _rounds(base, rs), None).model(-9, 30, 21, 18)
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


@pytest.mark.parametrize("rounds", [(2, 2), (3, 1)])
def test_rounds_local_coordinate_closed_form(rounds):
    # F = c_in x + u/H - 2 v/H (window-local coordinates u, v): each window
    # runs its own trajectory through a round, then the windows are blended;
    # written out per pixel and per covering window
    st = _rounds(synth.config1_stack(test_denoiser=3), rounds)
    lv = st["level"][0]
    H, s, K_ = lv["window"], lv["stride"], lv["steps"]
    y0, x0, h, w = -23, 40, 19, 21
    got = S.World(5, st, None).model(y0, x0, h, w)
    sig = Sc.sigmas(K_, lv["sigma_max"], lv["sigma_min"], lv["rho"])
    w1 = Sc.weight_1d(H, 1e-3)
    Y = np.arange(y0, y0 + h)[:, None] + np.zeros((1, w), dtype=np.int64)
    X = np.arange(x0, x0 + w)[None, :] + np.zeros((h, 1), dtype=np.int64)
    noise = [N.normal_region(5, 0, j, x0, y0, w, h).astype(np.float64) for j in range(K_)]
    J = sig[0] * noise[0]
    j0 = 0
    for m in rounds:
        num = np.zeros((h, w))
        den = np.zeros((h, w))
        for di in (0, 1):
            for dj in (0, 1):
                u = Y - (Y // s - di) * s
                v = X - (X // s - dj) * s
                ww = w1[u] * w1[v]
                g = u / H - 2.0 * v / H
                x = J.copy()
                for j in range(j0, j0 + m):
                    cs, co, ci = Sc.edm_coeffs(sig[j], lv["sigma_data"])
                    x = cs * x + co * (ci * x + g)
                    if j + 1 < K_:
                        x = x + sig[j + 1] * noise[j + 1]
                num += ww * x
                den += ww
        J = num / den
        j0 += m
    assert np.max(np.abs(got - J)) < 1e-12 * np.max(np.abs(J))


def _rounds_by_pixel(lv, rounds, seed, rect, F):
    """Blending only at round ends, written out per pixel and per covering
    window: each of the 2 x 2 windows over a pixel runs its own trajectory
    x <- c_skip x + c_out F(c_in x, g) + sigma_{j+1} N through the round, g
    the window-local coordinate term u/H - 2 v/H."""
    H, s, K_ = lv["window"], lv["stride"], lv["steps"]
    y0, x0, h, w = rect
    sig = Sc.sigmas(K_, lv["sigma_max"], lv["sigma_min"], lv["rho"])
    w1 = Sc.weight_1d(H, 1e-3)
    Y = np.arange(y0, y0 + h)[:, None] + np.zeros((1, w), dtype=np.int64)
    X = np.arange(x0, x0 + w)[None, :] + np.zeros((h, 1), dtype=np.int64)
    noise = [N.normal_region(seed, 0, j, x0, y0, w, h).astype(np.float64) for j in range(K_)]
    J = sig[0] * noise[0]
    j0 = 0
    for m in rounds:
        num = np.zeros((h, w))
        den = np.zeros((h, w))
        for di in (0, 1):
            for dj in (0, 1):
                u = Y - (Y // s - di) * s
                v = X - (X // s - dj) * s
                ww = w1[u] * w1[v]
                g = u / H - 2.0 * v / H
                x = J.copy()
                for j in range(j0, j0 + m):
                    cs, co, ci = Sc.edm_coeffs(sig[j], lv["sigma_data"])
                    x = cs * x + co * F(ci * x, g)
                    if j + 1 < K_:
                        x = x + sig[j + 1] * noise[j + 1]
                num += ww * x
                den += ww
        J = num / den
        j0 += m
    return J


@pytest.mark.parametrize("rounds", [(2, 2), (3, 1)])
def test_rounds_nonlinear_local_denoiser_closed_form(monkeypatch, rounds):
    # With a denoiser affine in x (the test denoisers), blending after every
    # step and blending at round ends agree: the blend is a normalised linear
    # combination, and it commutes with affine maps whose coefficients all
    # windows share.  A denoiser nonlinear in x and dependent on the window,
    # F = tanh(c_in x) + u/H - 2 v/H, tells the two apart.
    def nonlinear_local(kind, x):
        B, C, H, W = x.shape
        u = np.arange(H, dtype=np.float64)[:, None] / H
        v = np.arange(W, dtype=np.float64)[None, :] / W
        return np.tanh(x.sum(axis=1, keepdims=True)) + (u - 2.0 * v)[None, None]
    monkeypatch.setattr(U, "test_denoiser", nonlinear_local)
    st = _rounds(synth.config1_stack(test_denoiser=3), rounds)
    lv = st["level"][0]
    rect = (-23, 40, 19, 21)
    got = S.World(5, st, None).model(rect[0], rect[1], rect[2], rect[3])
    F = lambda xin, g: np.tanh(xin) + g   # noqa: E731
    ref = _rounds_by_pixel(lv, rounds, 5, rect, F)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    every = _rounds_by_pixel(lv, (1,) * lv["steps"], 5, rect, F)
    assert np.max(np.abs(every - ref)) > 1e-4 * np.max(np.abs(ref))


def test_rounds_lazy_equals_eager_and_cone_counts():
    st = _rounds(synth.config1_stack(), (2, 2))
    wts = _weights(st)
    lz = S.World(0, st, wts)
    lazy = lz.model(0, 0, 32, 32)
    eager = S.eager_world_model(0, st, wts, 0, 0, 32, 32)
    assert np.max(np.abs(lazy - eager)) <= 1e-12 * np.max(np.abs(eager))
    # two rounds: the cone of a 2-step sampler, each window run for 2 steps
    counts = K.cone_window_counts(0, 0, 32, 32, 32, 16, 2)
    assert counts == [(2 + 1) ** 2, (2 + 3) ** 2]
    assert lz.levels[0].phi_calls == 2 * sum(counts)



# ----------------------------------------------------------- conditioning and AutoGuidance

def _cond_setup(w, steps=1, z=(0.5, -1.0, 0.25, 2.0), amp=0.3):
    st = synth.with_steps(synth.conditioned(synth.config1_stack(), dim=4, z=z, amp=amp, guidance=w), steps)
    lv = st["level"][0]
    shapes = [s for _, s in U.param_shapes(lv)]
    main = synth.weights(shapes, 0, 0)
    guide = synth.guide_weights(main, shapes, 0)
    return st, main, guide


def test_guidance_is_affine_in_the_scale_for_one_step():
    # one blended step: J_1 = c_skip J_0 + c_out blend(F_g + w (F_m - F_g)),
    # so J_1(w) = (1 - w) J_1(guide) + w J_1(main) exactly (blending is linear)
    rect = (-9, 5, 20, 23)
    st2, main, guide = _cond_setup(2.15)
    got = S.World(4, st2, [main], guide_weights=[guide]).model(*rect)
    st0, _, _ = _cond_setup(0.0)
    j_main = S.World(4, st0, [main]).model(*rect)
    j_guide = S.World(4, st0, [guide]).model(*rect)
    ref = (1 - 2.15) * j_guide + 2.15 * j_main
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # w = 1 is the main network alone
    st1, _, _ = _cond_setup(1.0)
    j1 = S.World(4, st1, [main], guide_weights=[guide]).model(*rect)
    assert np.max(np.abs(j1 - j_main)) <= 1e-12 * np.max(np.abs(j_main))


def test_zero_conditioning_equals_the_unconditioned_network():
    # z = 0 and amp = 0 give y_i = 0, so E y_i = 0 whatever E is
    st, main, _ = _cond_setup(0.0, steps=2, z=(0.0, 0.0, 0.0, 0.0), amp=0.0)
    plain = synth.with_steps(synth.config1_stack(), 2)
    n_plain = sum(int(np.prod(s)) for _, s in U.param_shapes(plain["level"][0]))
    rect = (3, -7, 17, 19)
    a = S.World(1, st, [main]).model(*rect)
    b = S.World(1, plain, [main[:n_plain]]).model(*rect)
    assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    # with a non-zero vector the result moves, and differs between windows
    st_c, _, _ = _cond_setup(0.0, steps=2)
    c = S.World(1, st_c, [main]).model(*rect)
    assert np.max(np.abs(c - b)) > 1e-3 * np.max(np.abs(b))
    lvl = S.World(1, st_c, [main]).levels[0]
    assert not np.allclose(lvl.cond_vector(0, 0), lvl.cond_vector(0, 1))
