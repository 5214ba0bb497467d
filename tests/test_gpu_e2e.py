"""End-to-end parity of the sampling path at the full network widths of the
2-level stack (coarse 64/128/128, fine 64/128/256/256 with attention,
128-pixel windows at stride 64), shortened to 2 blended steps so that the
FP64 oracle can evaluate the whole dependency cone (40 windows)."""
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


def test_two_level_full_width_plain_bf16(case):
    # Plain BF16 operands.  With 2 steps (sigma 80 then 0.02) the result is
    # almost exactly one network evaluation, 0.5 F(noise), so the network's
    # rounding error reaches sigma_out undamped: about 0.9% rms and 4% at the
    # largest of the 4096 pixels (operand rounding 2^-9 through ~25
    # convolutions).  That exceeds the 2e-2 sigma_out target on this
    # worst-case cone, which is why IDF_BF16X3 exists; here the measured
    # error is checked against the bound the bfloat16 arithmetic implies.
    idf, st, wts, rect, ref = case
    W = idf.World(0, st, wts, precision="bf16")
    got = W.query(*rect).astype(np.float64)
    W.close()
    sig = ref.std()
    d = got - ref
    rms, mx = float(np.sqrt(np.mean(d * d))) / sig, float(np.max(np.abs(d))) / sig
    print(f"bf16: rms {rms:.3e} sigma_out, max {mx:.3e} sigma_out")
    assert rms <= 1.5e-2 and mx <= 6e-2


def test_two_level_full_width_four_steps():
    # Four blended steps (sigma 80, 12.7, 1.03, 0.02) through the same full
    # width stack: a deeper cone (120 fine windows) than the two-step case,
    # TF32 and BF16X3 against the stated 2e-2 sigma_out bound
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st = synth.config2_stack(steps=4)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    rect = (0, 0, 64, 64)
    ref = OS.World(0, st, wts).model(rect[1], rect[0], rect[3], rect[2])
    sig = ref.std()
    for precision in ("tf32", "bf16x3"):
        W = idf.World(0, st, wts, precision=precision)
        got = W.query(*rect).astype(np.float64)
        W.close()
        err = np.max(np.abs(got - ref))
        print(f"4 steps {precision}: max abs err {err / sig:.3e} sigma_out")
        assert err <= 2e-2 * sig


def test_tf32_against_bf16x3_twenty_steps():
    # The full 20-step configuration on a 256 x 256 crop (about 18k fine and
    # 17k coarse window evaluations: beyond the FP64 oracle's reach in a
    # test).  BF16X3 matches the oracle to ~1e-4 sigma_out where the oracle
    # can check it, so the TF32 - BF16X3 difference measures TF32's error
    # here to within that.
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st = synth.config2_stack(steps=20)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    rect = (1920, 1920, 256, 256)
    out = {}
    for precision in ("bf16x3", "tf32"):
        W = idf.World(0, st, wts, precision=precision)
        out[precision] = W.query(*rect).astype(np.float64)
        W.close()
    sig = out["bf16x3"].std()
    d = out["tf32"] - out["bf16x3"]
    mx, rms = float(np.max(np.abs(d))) / sig, float(np.sqrt(np.mean(d * d))) / sig
    print(f"20 steps, 256^2 crop: tf32 - bf16x3 max {mx:.3e} rms {rms:.3e} sigma_out (sigma_out {sig:.4f})")
    assert mx <= 1.9e-2
