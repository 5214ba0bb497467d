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


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("bf16", 2e-2)])
def test_two_level_full_width(case, precision, tol):
    idf, st, wts, rect, ref = case
    W = idf.World(0, st, wts, precision=precision)
    got = W.query(*rect).astype(np.float64)
    W.close()
    sig = ref.std()
    err = np.max(np.abs(got - ref))
    print(f"{precision}: max abs err {err:.3e} = {err / sig:.3e} sigma_out (sigma_out {sig:.4f})")
    assert err <= tol * sig
