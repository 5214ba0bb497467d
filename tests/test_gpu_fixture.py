"""Earth-scale decode with a given low band: a single-level stack whose level
(the 16-channel UNet of the 32x32-window configuration) generates the
residual band and whose low band is a periodic fixture of signed-sqrt
elevations, decoded to metres on the GPU and compared with the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import sampler as OS
from oracle import unet as OU

pytestmark = pytest.mark.gpu


def test_metres_with_fbm_fixture_match_oracle():
    import paper_2512_08309_gb300 as idf
    idf.lib()
    # a small periodic fBm fixture (64 low-resolution px = 512 px period)
    # spanning the signed square roots of [-11000, 9000] metres
    fx = synth.fbm_lowband(64, beta=2.2, seed=0)
    st = synth.config4_stack(fx, steps=4)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    # the query crosses the fixture's period boundary (x = 512) and y = 0
    rect = (480, -24, 64, 48)   # x0, y0, w, h
    W = idf.World(0, st, wts, precision="fp32")
    got = W.query(*rect, kind=idf.IDF_OUT_METRES).astype(np.float64)
    Hm = W.query(*rect, kind=idf.IDF_OUT_MODEL).astype(np.float64)
    W.close()
    ow = OS.World(0, st, wts)
    ref = ow.metres(rect[1], rect[0], rect[3], rect[2])
    Href = ow.model(rect[1], rect[0], rect[3], rect[2])
    # bound from the arithmetic: the FP32 network path is within 1e-4
    # sigma_H of the oracle (its own bound), so v = up(l^) + res_scale H is
    # off by at most res_scale 1e-4 sigma_H plus the float32 rounding of the
    # decode chain (a few hundred roundings of values of size |v|: 1e-5 |v|);
    # metres = sign(v) v^2 then differ by at most 2 |v| dv + dv^2
    sig_h = Href.std()
    assert np.max(np.abs(Hm - Href)) <= 1e-4 * sig_h
    v = np.sign(ref) * np.sqrt(np.abs(ref))
    dv = 1.5 * 1e-4 * sig_h + 1e-5 * np.abs(v)
    bound = 2 * np.abs(v) * dv + dv * dv
    err = np.abs(got - ref)
    print(f"metres: max |err| {err.max():.3e} m over |m| <= {np.abs(ref).max():.0f} m; "
          f"max err/bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)
