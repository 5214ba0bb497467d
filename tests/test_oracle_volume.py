"""Pins of the Z^3 oracle: closed forms of the test denoisers, lazy Alg. 1 ==
eager Eq. 1, the 3-D network against torch.nn.functional (FP64), the cone's
window counts, and the volume noise's distribution."""
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as TF

import synth
from oracle import kappa as K
from oracle import noise as N
from oracle import schedule as Sc
from oracle import volume as V


def _closed_form(desc, seed, box, F_of_J):
    z0, y0, x0, d, h, w = box
    sig = Sc.sigmas(desc["steps"], desc["sigma_max"], desc["sigma_min"], desc["rho"])
    J = sig[0] * V.normal3_box(seed, 0, 0, z0, y0, x0, d, h, w).astype(np.float64)
    for k in range(desc["steps"]):
        cs, co, ci = Sc.edm_coeffs(sig[k], desc["sigma_data"])
        J = cs * J + co * F_of_J(J, ci)
        if k + 1 < desc["steps"]:
            J = J + sig[k + 1] * V.normal3_box(seed, 0, k + 1, z0, y0, x0, d, h, w)
    return J


@pytest.mark.parametrize("td", [1, 2])
def test_pixel_local_denoisers_closed_form(td):
    desc = synth.volume_desc(test_denoiser=td)
    box = (-5, 9, -13, 7, 6, 9)
    got = V.VolumeLevel(3, desc).final(*box)
    F = (lambda J, ci: 0.5) if td == 1 else (lambda J, ci: ci * J)
    ref = _closed_form(desc, 3, box, F)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_local_coordinate_denoiser_closed_form():
    # F = c_in J + u/H - 2 v/H + 3 w/H: the blend adds the weighted mean of
    # the window-local coordinate term over the r^3 windows covering a voxel
    desc = synth.volume_desc(test_denoiser=3)
    H, s = desc["window"], desc["stride"]
    box = (4, -11, 6, 5, 7, 6)
    got = V.VolumeLevel(1, desc).final(*box)
    w1 = Sc.weight_1d(H, 1e-3)
    z0, y0, x0, d, h, w = box
    g = np.zeros((d, h, w))
    for a in range(d):
        for b in range(h):
            for c in range(w):
                Z, Y, X = z0 + a, y0 + b, x0 + c
                num = den = 0.0
                for i in range(Z // s - 1, Z // s + 1):
                    for j in range(Y // s - 1, Y // s + 1):
                        for l in range(X // s - 1, X // s + 1):
                            u, v, t = Z - i * s, Y - j * s, X - l * s
                            ww = w1[u] * w1[v] * w1[t]
                            num += ww * (u / H - 2.0 * v / H + 3.0 * t / H)
                            den += ww
                g[a, b, c] = num / den
    ref = _closed_form(desc, 1, box, lambda J, ci: ci * J + g)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_network_matches_torch():
    desc = synth.volume_desc()
    p = V.unpack(desc, synth.volume_weights(desc))
    x = np.random.default_rng(0).standard_normal((2, 1, 16, 16, 16))
    t = {k: torch.from_numpy(v) for k, v in p.items()}
    h = TF.conv3d(torch.from_numpy(x), t["conv1"], padding=1)
    h = TF.silu(TF.group_norm(h, 4, eps=1e-5))
    ref = TF.conv3d(h, t["conv2"], padding=1).numpy()
    got = V.forward(desc, p, x)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_lazy_equals_eager_and_cone_count():
    desc = synth.volume_desc(steps=2)
    wts = synth.volume_weights(desc)
    box = (0, 8, -8, 8, 8, 8)   # one aligned tile
    lz = V.VolumeLevel(0, desc, wts)
    a = lz.final(*box)
    b = V.eager_volume(0, desc, wts, *box)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    # Lemma 4 on Z^3: a cold query of an n^3-tile box evaluates
    # sum_k (n + 2k + 1)^3 windows (n = 1, two steps: 8 + 64)
    assert lz.phi_calls == sum((1 + 2 * k + 1) ** 3 for k in range(2))
    assert len(V.kappa3(0, 8, -8, 8, 8, 8, 16, 8)) == 8


def test_volume_noise_is_standard_normal_and_apart_from_2d():
    z = V.normal3_box(5, 0, 1, -40, 0, 7, 40, 50, 60).astype(np.float64).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n) and abs(z.var() - 1) < 5 * math.sqrt(2 / n)
    from scipy import stats
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the 2-D seed function at the same (x, y) and step differs
    a = V.normal3(5, 0, 1, np.arange(100), 3, 0)
    b = N.normal(5, 0, 1, np.arange(100), 3)
    assert not np.any(a == b)
