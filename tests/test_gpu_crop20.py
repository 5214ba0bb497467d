"""The full 20-step configuration of the 2-level stack against the FP64
oracle, element by element, on 256 x 256 crops: at (1920, 1920), and at
(-128, -128) across the origin (negative tile indices and their floor
division at the full width and step count).

The expected values were written once by tests/golden/make_config2_crop.py,
which calls only the oracle (Eq. 1 brute force over the crop's whole
dependency cone, ~35k window evaluations in FP64): the fine level's J_K over
the crop, the coarse level's J_K over the low-band rect the decode reads,
and the decoded metres.  Bounds: 1e-4 sigma_out (FP32) and 2e-2 sigma_out
(the tensor-core precisions), sigma_out the population std of the oracle's
values over the checked rect.  Metres are held per pixel to the bound that
follows from the model-space bounds: the decode v = up(blur(down(up(l) +
h))) + h is a convex combination at every stage, so |dv| <= low_scale e_L +
2 res_scale e_H, and metres = sign(v) v^2 gives |dm| <= 2 |v| dv + dv^2."""
import os

import numpy as np
import pytest

import synth
from oracle import unet as OU

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FIXTURES = ["config2_crop_k20.npz", "config2_crop_k20_origin.npz"]

BF16_MISS = ("plain BF16 misses 2e-2 sigma_out at the full 20 steps: measured at (1920, 1920) 7.8e-2 "
             "sigma_out (fine), 2.4e-2 (coarse), 2.2 m in metres, and at (-128, -128) 5.3e-2 (fine), 1.2e-2 "
             "(coarse), 0.54 m; bfloat16 operand rounding through ~25 convolutions per "
             "network evaluation, compounded over the 20 evaluations of the chain (1.9e-2 at 4 steps)")


@pytest.fixture(scope="module", params=FIXTURES)
def fix(request):
    path = os.path.join(GOLDEN, request.param)
    if not os.path.exists(path):
        pytest.skip(f"the oracle fixture {request.param} has not been written (tests/golden/make_config2_crop.py)")
    d = np.load(path)
    st = synth.config2_stack(steps=int(d["steps"]))
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    import paper_2512_08309_gb300 as idf
    idf.lib()
    return idf, d, st, wts


@pytest.mark.parametrize("precision,tol", [
    ("fp32", 1e-4), ("tf32", 2e-2), ("bf16x3", 2e-2),
    pytest.param("bf16", 2e-2, marks=pytest.mark.xfail(reason=BF16_MISS, strict=False)),
])
def test_twenty_steps_against_oracle(fix, precision, tol):
    idf, d, st, wts = fix
    x0, y0, w, h = (int(v) for v in d["crop"])
    ref_m, ref_v = d["model"].astype(np.float64), d["metres"].astype(np.float64)
    sig_m = float(d["sigma_model"])
    W = idf.World(int(d["seed"]), st, wts, precision=precision)
    got_m = W.query(x0, y0, w, h).astype(np.float64)
    got_v = W.query(x0, y0, w, h, kind=idf.IDF_OUT_METRES).astype(np.float64)
    W.close()
    # the coarse level alone (same seed, level index 0, weights): its J_K over
    # the low-band rect the decode reads
    coarse = synth.stack([st["level"][0]])
    Wc = idf.World(int(d["seed"]), coarse, [wts[0]], precision=precision)
    lx0, ly0, lw, lh = (int(v) for v in d["low_rect"])
    got_l = Wc.query(lx0, ly0, lw, lh).astype(np.float64)
    Wc.close()
    ref_l, sig_l = d["low"].astype(np.float64), float(d["sigma_low"])
    e_m = float(np.max(np.abs(got_m - ref_m)))
    e_l = float(np.max(np.abs(got_l - ref_l)))
    dv = st["low_scale"] * tol * sig_l + 2.0 * st["res_scale"] * tol * sig_m
    bound = 2.0 * np.sqrt(np.abs(ref_v)) * dv + dv * dv + 1e-5 * np.abs(ref_v) + 1e-3
    e_v = np.abs(got_v - ref_v)
    print(f"{precision}: fine {e_m / sig_m:.3e} sigma_out, coarse {e_l / sig_l:.3e} sigma_out, "
          f"metres max {e_v.max():.4f} m (worst {np.max(e_v / bound):.3f} of its bound; "
          f"metres range {ref_v.min():.1f}..{ref_v.max():.1f})")
    assert e_m <= tol * sig_m
    assert e_l <= tol * sig_l
    assert np.all(e_v <= bound)
