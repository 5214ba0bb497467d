"""GroupNorm + SiLU inside the TF32 tensor-core convolutions' operand path
(the option groupnorm_in_conv; off by default because it measured slower).

The fused path applies, in shared memory, the same arithmetic as the
separate GroupNorm apply pass ((x - mean) * rstd, SiLU with the fast
exponential and division, tf32 rounding to nearest with ties away) with the
same statistics kernels, so it must give the separate path's result bit for
bit: per UNet window batch (ResBlocks, the attention block's normalisation,
the half-resolution decoder blocks with the concat's statistics and the
rounded shortcut operands) and through whole queries."""
import numpy as np
import pytest

import synth
from oracle import unet as OU

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def idf():
    import paper_2512_08309_gb300 as m
    m.lib()
    return m


def _weights(st):
    return [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]


@pytest.mark.parametrize("li", [0, 1])
def test_unet_fused_equals_separate(idf, li):
    st = synth.config2_stack()
    wts = _weights(st)
    lv = st["level"][li]
    n = 5
    x = synth.window_batch(n, lv["in_ch"], lv["window"], seed=11 + li)
    xd = torch.from_numpy(x).cuda()
    outs = []
    for fused in (True, False):
        W = idf.World(0, st, wts, precision="tf32", max_batch=3, groupnorm_in_conv=fused)
        yd = torch.empty((n, 1, lv["window"], lv["window"]), device="cuda")
        W.unet_forward(li, xd.data_ptr(), n, yd.data_ptr())
        torch.cuda.synchronize()
        W.close()
        outs.append(yd.cpu().numpy())
    assert np.all(np.isfinite(outs[0]))
    assert np.array_equal(outs[0], outs[1])


def test_query_fused_equals_separate(idf):
    st = synth.config2_stack(steps=2)
    wts = _weights(st)
    rect = (-70, 33, 96, 80)
    res = []
    for fused in (True, False):
        W = idf.World(0, st, wts, precision="tf32", groupnorm_in_conv=fused)
        res.append((W.query(*rect), W.query(*rect, kind=idf.IDF_OUT_METRES)))
        W.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])


def test_wait_budget_option_is_accepted(idf):
    # a generous explicit budget behaves like the default
    st = synth.config2_stack(steps=2)
    wts = _weights(st)
    a = idf.World(0, st, wts, precision="tf32", wait_budget_cycles=4_000_000_000)
    b = idf.World(0, st, wts, precision="tf32")
    assert np.array_equal(a.query(0, 0, 64, 64), b.query(0, 0, 64, 64))
    a.close()
    b.close()
