"""The tensor-core convolutions' tile-shape autotuner: every valid shape
(BN output channels, MT M tiles per unit, staging per kernel row or per
tap) gives the same result bit for bit, so a world that times them and keeps
the fastest answers exactly as a world with the built-in shapes."""
import numpy as np
import pytest

import synth
from oracle import unet as OU

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["tf32", "bf16x3"])
def test_autotuned_world_equals_builtin_shapes(precision):
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st = synth.config2_stack(steps=2)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    rect = (-64, 32, 96, 80)
    A = idf.World(0, st, wts, precision=precision, autotune=True)
    a = A.query(*rect, kind=idf.IDF_OUT_METRES)
    a2 = A.query(rect[0] + 640, rect[1], rect[2], rect[3])   # uses the tuned shapes
    at = A.stats()["autotune"]
    A.close()
    B = idf.World(0, st, wts, precision=precision)
    b = B.query(*rect, kind=idf.IDF_OUT_METRES)
    b2 = B.query(rect[0] + 640, rect[1], rect[2], rect[3])
    B.close()
    print(f"{precision}: {at['tuned']} layer classes tuned, {at['changed']} with a shape other than the built-in")
    assert at["tuned"] > 0
    assert np.array_equal(a, b) and np.array_equal(a2, b2)
