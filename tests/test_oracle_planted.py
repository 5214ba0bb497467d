"""The oracle's pins have the power to catch its plausible mistakes.

Each case plants one mistake in the oracle (on the CPU, for the duration of
the case: a dropped term, a wrong sign, an off-by-one index, a transposed
operand, a shifted grid) and runs the pins that guard that function; at
least one of them must fail with an assertion.  Every pin is called with
arguments that its own test file runs it with, where it passes on the
oracle as it stands.  A pin set that let one of these mistakes through
would not be evidence that the oracle computes what the paper defines."""
import types

import numpy as np
import pytest

import test_oracle_kappa as TK
import test_oracle_laplacian as TL
import test_oracle_noise as TN
import test_oracle_sampler as TS
import test_oracle_student as TST
import test_oracle_unet as TU
import test_oracle_volume as TV
import synth
from oracle import kappa as K
from oracle import laplacian as L
from oracle import noise as N
from oracle import sampler as S
from oracle import schedule as Sc
from oracle import student as OST
from oracle import unet as U
from oracle import volume as V

_kappa_1d, _cone, _philox, _ln, _cos, _normal = (K.kappa_1d, K.cone_window_counts, N.philox4x32_10, N.ln_f32,
                                                 N.cos2pi_f32, N.normal)
_sigmas, _edm = Sc.sigmas, Sc.edm_coeffs
_conv, _gn, _silu, _pool, _up2, _attn, _cbias = (U.conv, U.group_norm, U.silu, U.avg_pool2, U.up2, U.attention,
                                                 U.cond_bias)
_taps, _down = L.blur_taps, L.down_mean
_lossg = OST.loss_and_grad
_kappa3, _conv3 = V.kappa3, V.conv3
_net, _init = S._LevelCommon.net, S._LevelCommon.__init__


def _shim(module, **over):
    """A stand-in for one of the oracle's modules with some names replaced."""
    ns = types.SimpleNamespace(**{k: getattr(module, k) for k in dir(module) if not k.startswith("__")})
    for k, v in over.items():
        setattr(ns, k, v)
    return ns


def _kappa_floor(start, stop, size, stride, offset=0):
    # first window index rounded down instead of up
    if stop <= start:
        return None
    i_min = (start - offset - size + 1) // stride
    i_max = (stop - 1 - offset) // stride
    return None if i_min > i_max else (i_min, i_max)


def _up_index_shifted(c0, n, f):
    # bilinear weights of corner-aligned instead of half-pixel-centred pixels
    c = np.arange(c0, c0 + n, dtype=np.int64)
    lo = c // f
    return lo, (c - lo * f) / float(f)


def _weight_1d_centre_off(size, eps):
    c = size / 2.0
    u = np.arange(size, dtype=np.float64)
    return 1.0 - (1.0 - eps) * np.abs(u - c) / c


def _adamw_no_bias_correction(w, g, m, v, t, lr=2e-4, b1=0.9, b2=0.999, eps=1e-8, wd=0.01):
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    return w - lr * (m / (np.sqrt(v) + eps) + wd * w), m, v


def _denoise_side_scaled(lv, p, x, sigma):
    # c_in applied to the side channels as well as to the state
    import torch
    c_skip, c_out, c_in = Sc.edm_coeffs(float(sigma), float(lv["sigma_data"]))
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64))
    if xt.dim() == 3:
        xt = xt[:, None]
    return c_skip * xt[:, :1] + c_out * OST.forward_torch(lv, p, c_in * xt)


def _cond_rounded(self, y0, x0, h, w):
    # the parent pixel of a fine pixel taken by rounding instead of flooring
    f = self.scale
    ys, xs = (np.arange(y0, y0 + h) + f // 2) // f, (np.arange(x0, x0 + w) + f // 2) // f
    P = self.parent.final(ys[0], xs[0], ys[-1] - ys[0] + 1, xs[-1] - xs[0] + 1)
    return P[np.ix_(ys - ys[0], xs - xs[0])]


def _net_roles_swapped(self, xin, ys):
    # AutoGuidance with the main and guide networks in each other's place
    if self.guide is None:
        return _net(self, xin, ys)
    self.params, self.guide = self.guide, self.params
    try:
        return _net(self, xin, ys)
    finally:
        self.params, self.guide = self.guide, self.params


def _init_blend_every_step(self, *a, **k):
    # the round grouping ignored: Eq. 2 after every sampler step
    _init(self, *a, **k)
    self.round_steps, self.R, self.round_start = [1] * self.K, self.K, list(range(self.K))


def _rounds_pin():
    with pytest.MonkeyPatch.context() as mp:
        TS.test_rounds_nonlinear_local_denoiser_closed_form(mp, (2, 2))


ATTN_LV = synth.level(levels=3, channels=(8, 16, 16), in_ch=2, attn_at_bottom=1, attn_heads=2, window=16)
SMALL_LV = synth.config1_stack()["level"][0]


def _set(mod, name, fn):
    return lambda mp: mp.setattr(mod, name, fn)


# (id, plant, pins)
CASES = [
    # kappa (Alg. 3) and the cone counts (Lemma 4)
    ("kappa_first_window_floor", _set(K, "kappa_1d", _kappa_floor), [TK.test_kappa_brute_force]),
    ("kappa_last_window_dropped",
     _set(K, "kappa_1d", lambda a, b, s, t, o=0: (lambda r: r and (r[0], r[1] - 1))(_kappa_1d(a, b, s, t, o))),
     [TK.test_kappa_brute_force]),
    ("cone_counts_one_extra_ring", _set(K, "cone_window_counts", lambda *a, **k: [c + 1 for c in _cone(*a, **k)]),
     [TK.test_cone_counts_closed_form]),
    # noise G (Philox4x32-10, Box-Muller)
    ("philox_key_words_swapped",
     _set(N, "philox4x32_10", lambda c0, c1, c2, c3, k0, k1: _philox(c0, c1, c2, c3, k1, k0)),
     [lambda: TN.test_philox_known_answers(*TN.KAT[2])]),
    ("philox_counter_words_swapped",
     _set(N, "philox4x32_10", lambda c0, c1, c2, c3, k0, k1: _philox(c1, c0, c2, c3, k0, k1)),
     [lambda: TN.test_philox_known_answers(*TN.KAT[2])]),
    ("ln_of_one_minus_u",
     _set(N, "ln_f32", lambda u: _ln(np.float32(1.0) - np.asarray(u, np.float32) + np.float32(2.0 ** -24))),
     [TN.test_ln_f32_whole_domain]),
    ("sin_for_cos", _set(N, "cos2pi_f32", lambda k: _cos((np.asarray(k, np.int64) + 3 * (1 << 22)) % (1 << 24))),
     [TN.test_cos2pi_f32_whole_domain]),
    ("noise_x_y_transposed", _set(N, "normal", lambda seed, level, step, x, y: _normal(seed, level, step, y, x)),
     [TN.test_normal_counter_layout]),
    ("noise_ignores_level", _set(N, "normal", lambda seed, level, step, x, y: _normal(seed, 0, step, x, y)),
     [TN.test_normal_decorrelated_across_step_level_seed]),
    # schedule and preconditioning (EDM)
    ("sigmas_without_rho", _set(Sc, "sigmas", lambda n, a, b, rho: _sigmas(n, a, b, 1.0)), [TS.test_sigma_schedule]),
    ("c_skip_c_out_swapped", _set(Sc, "edm_coeffs", lambda s, sd: (lambda c: (c[1], c[0], c[2]))(_edm(s, sd))),
     [TS.test_edm_identity]),
    ("weight_window_centre_off_by_half", _set(Sc, "weight_1d", _weight_1d_centre_off),
     [TS.test_weight_window_and_denominator]),
    # the sampler (Eq. 1, Eq. 2, Alg. 1)
    ("renoise_step_off_by_one",
     lambda mp: mp.setattr(S, "N_", _shim(N, normal_region=lambda sd, lv, st, *a: N.normal_region(
         sd, lv, st + 1 if st > 0 else 0, *a))),
     [lambda: TS.test_constant_and_identity_denoisers_closed_form(1)]),
    ("input_preconditioning_dropped",
     lambda mp: mp.setattr(S, "S_", _shim(Sc, edm_coeffs=lambda s, sd: (lambda c: (c[0], c[1], 1.0))(_edm(s, sd)))),
     [lambda: TS.test_constant_and_identity_denoisers_closed_form(2)]),
    ("flat_blend_window",
     lambda mp: mp.setattr(S, "S_", _shim(Sc, weight_2d=lambda size, eps: np.ones((size, size)))),
     [TS.test_local_coordinate_denoiser_closed_form]),
    ("conditioning_parent_pixel_rounded", _set(S._LevelCommon, "cond", _cond_rounded),
     [TS.test_conditioning_closed_form_two_level]),
    ("guidance_roles_swapped", _set(S._LevelCommon, "net", _net_roles_swapped),
     [TS.test_guidance_is_affine_in_the_scale_for_one_step]),
    ("rounds_ignored", _set(S._LevelCommon, "__init__", _init_blend_every_step),
     [_rounds_pin]),
    # the window denoiser (UNet)
    ("conv_kernel_flipped", _set(U, "conv", lambda x, w: _conv(x, w[:, :, ::-1, ::-1])),
     [TU.test_conv_is_cross_correlation]),
    ("groupnorm_one_group", _set(U, "group_norm", lambda x, g: _gn(x, 1)),
     [lambda: TU.test_unet_matches_torch_functional(SMALL_LV)]),
    ("silu_sign", _set(U, "silu", lambda x: x - _silu(x)), [lambda: TU.test_unet_matches_torch_functional(SMALL_LV)]),
    ("pool_grid_shifted", _set(U, "avg_pool2", lambda x: _pool(np.roll(x, 1, axis=3))),
     [lambda: TU.test_unet_matches_torch_functional(SMALL_LV)]),
    ("upsample_grid_shifted", _set(U, "up2", lambda x: np.roll(_up2(x), 1, axis=2)),
     [lambda: TU.test_unet_matches_torch_functional(SMALL_LV)]),
    ("attention_residual_dropped", _set(U, "attention", lambda x, p, g, h: _attn(x, p, g, h) - x),
     [lambda: TU.test_unet_matches_torch_functional(ATTN_LV)]),
    ("conditioning_bias_sign", _set(U, "cond_bias", lambda p, y: -_cbias(p, y)),
     [TU.test_conditioning_bias_matches_torch_linear]),
    # the Laplacian decode and the signed square
    ("plain_square", _set(L, "signed_square", lambda x: np.asarray(x, np.float64) ** 2), [TL.test_signed_sqrt_pair]),
    ("blur_sigma_wrong", _set(L, "blur_taps", lambda s, r: _taps(1.5 * s, r)), [TL.test_blur_taps]),
    ("up_weights_corner_aligned", _set(L, "_up_index", _up_index_shifted),
     [TL.test_up_weights_are_half_pixel_centred]),
    ("down_grid_shifted", _set(L, "down_mean", lambda P, f: _down(np.roll(P, 1, axis=1), f)),
     [TL.test_lowband_noise_gain_matches_impulse_response]),
    # the student
    ("gradient_sign", _set(OST, "loss_and_grad", lambda *a: (lambda r: (r[0], -r[1]))(_lossg(*a))),
     [TST.test_gradient_matches_central_differences]),
    ("adamw_without_bias_correction", _set(OST, "adamw", _adamw_no_bias_correction), [TST.test_adamw_step_by_hand]),
    ("side_channels_preconditioned", _set(OST, "_denoise", _denoise_side_scaled),
     [TST.test_side_channels_enter_unscaled_and_state_only_through_channel_zero]),
    # volumes on Z^3
    ("kappa3_last_window_dropped", _set(V, "kappa3", lambda *a: _kappa3(*a)[:-1]),
     [TV.test_local_coordinate_denoiser_closed_form]),
    ("conv3_kernel_flipped", _set(V, "conv3", lambda x, w: _conv3(x, w[:, :, ::-1, ::-1, ::-1])),
     [TV.test_network_matches_torch]),
]


@pytest.mark.parametrize("plant,pins", [c[1:] for c in CASES], ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(monkeypatch, plant, pins):
    plant(monkeypatch)
    caught = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught += 1
    assert caught, "no pin caught the planted mistake"

