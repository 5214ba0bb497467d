"""Persistent tile store: a later session of the same world reads finalized
tiles instead of recomputing their cones, with results bit for bit equal to
a cold world's; a store refuses another world."""
import os

import numpy as np
import pytest

import synth
from oracle import unet as OU

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def idf():
    import paper_2512_08309_gb300 as m
    m.lib()
    return m


def _setup():
    st = synth.small_hier_stack(steps=3)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    return st, wts


def test_store_session_resume(idf, tmp_path):
    st, wts = _setup()
    d = str(tmp_path / "tiles")
    rect, inner = (-40, 24, 96, 72), (-24, 40, 48, 32)
    A = idf.World(0, st, wts, precision="fp32")
    A.store_open(d, writable=True)
    a_m = A.query(*rect, kind=idf.IDF_OUT_METRES).copy()
    a_i = A.query(*inner).copy()
    sa = A.stats()["levels"]
    assert all(l["store_writes"] > 0 for l in sa)
    A.store_close()
    A.close()
    assert os.path.exists(os.path.join(d, "idf_store.manifest"))

    # a new session: the same queries are read from the store, nothing is evaluated
    B = idf.World(0, st, wts, precision="fp32")
    B.store_open(d, writable=False)
    assert np.array_equal(B.query(*rect, kind=idf.IDF_OUT_METRES), a_m)
    assert np.array_equal(B.query(*inner), a_i)
    sb = B.stats()["levels"]
    assert all(l["windows_evaluated"] == 0 for l in sb)
    assert all(l["store_reads"] > 0 for l in sb)
    # a region reaching beyond the stored tiles: computes the rest, and
    # equals a cold world bit for bit
    shifted = (rect[0] + 200, rect[1], rect[2], rect[3])
    got = B.query(*shifted, kind=idf.IDF_OUT_METRES)
    ev = [l["windows_evaluated"] for l in B.stats()["levels"]]
    B.store_close()
    B.close()
    C = idf.World(0, st, wts, precision="fp32")
    ref = C.query(*shifted, kind=idf.IDF_OUT_METRES)
    cold = [l["windows_evaluated"] for l in C.stats()["levels"]]
    C.close()
    assert np.array_equal(got, ref)
    assert sum(ev) < sum(cold)


def test_store_refuses_another_world(idf, tmp_path):
    st, wts = _setup()
    d = str(tmp_path / "tiles")
    A = idf.World(0, st, wts, precision="fp32")
    A.store_open(d, writable=True)
    A.query(0, 0, 16, 16)
    A.store_close()
    A.close()
    for seed, prec in ((1, "fp32"), (0, "bf16")):
        W = idf.World(seed, st, wts, precision=prec)
        with pytest.raises(idf.IdfError) as e:
            W.store_open(d, writable=False)
        assert e.value.status == idf.IDF_EINVAL
        W.close()
    W = idf.World(0, st, wts, precision="fp32")
    with pytest.raises(idf.IdfError):
        W.store_open(str(tmp_path / "absent"), writable=False)
    W.close()
