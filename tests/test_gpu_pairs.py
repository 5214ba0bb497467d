"""Tensor-core convolutions on CTA pairs (clusters of two CTAs, cta_group::2
products of M = 256): each CTA stages its own pixels and half of the weight
tile, and every output element gets the same products in the same K order as
on one CTA, so a world with pairs answers bit for bit as one without.  Checked
for the plain BF16 and TF32 networks of the 2-level stack, through whole
queries and through idf_unet_forward at batch sizes whose M tiles pair up
and whose do not (those fall back to one CTA)."""
import numpy as np
import pytest

import synth
from oracle import unet as OU

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _stack():
    st = synth.config2_stack(steps=2)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    return st, wts


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_pair_world_equals_single_cta_world(precision):
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st, wts = _stack()
    rects = [(-64, 32, 96, 80), (576, 2000, 130, 70)]
    out = {}
    for pairs in (True, False):
        W = idf.World(0, st, wts, precision=precision, max_batch=16, cta_pairs=pairs)
        out[pairs] = [W.query(*r, kind=idf.IDF_OUT_METRES) for r in rects]
        W.close()
    for a, b in zip(out[True], out[False]):
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
@pytest.mark.parametrize("level", [0, 1])
def test_pair_unet_forward_equals_single_cta(precision, level):
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st, wts = _stack()
    lv = st["level"][level]
    H, cin = lv["window"], lv["in_ch"]
    res = {}
    for pairs in (True, False):
        W = idf.World(0, st, wts, precision=precision, max_batch=8, cta_pairs=pairs)
        res[pairs] = []
        for n in (1, 2, 3, 8):
            g = torch.Generator().manual_seed(100 + n)
            x = torch.randn((n, cin, H, H), generator=g).cuda()
            y = torch.empty((n, 1, H, H), device="cuda")
            W.unet_forward(level, x.data_ptr(), n, y.data_ptr())
            torch.cuda.synchronize()
            res[pairs].append(y.cpu().numpy())
        s = W.stats()
        W.close()
        assert s["device_status"]["waits_expired"] == 0
    for a, b in zip(res[True], res[False]):
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b)
