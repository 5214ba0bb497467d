"""Failure detection end to end, injected from the host (no device fault,
no device wait is shortened or run out).

The tensor-core convolutions bound every wait and, when one runs out, set a
device status word; the conditioning gather sets a flag instead of reading
out of range.  Here the test writes those words from the host
(idf_debug_set_status) before a synchronizing query, so the library's own
paths that follow a real expiry or bounds violation run unchanged: the query
returns IDF_ETIMEOUT and the world is poisoned (IDF_EINTERNAL afterwards),
or the query returns IDF_EDEVICE_CHECK and the world stays usable.  A fresh
world on the same device then gives the correct result, so the CUDA context
survived."""
import numpy as np
import pytest

import synth
from oracle import unet as OU

pytestmark = pytest.mark.gpu

RECT = (0, 0, 64, 64)


@pytest.fixture(scope="module")
def idf():
    import paper_2512_08309_gb300 as m
    m.lib()
    return m


def _stack():
    st = synth.config2_stack(steps=2)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    return st, wts


def test_wait_expiry_status_poisons_the_world(idf):
    st, wts = _stack()
    W = idf.World(0, st, wts, precision="tf32")
    good = W.query(*RECT).copy()
    W.cache_clear()
    W.debug_set_status(0, 1)
    with pytest.raises(idf.IdfError) as e:
        W.query(*RECT)
    assert e.value.status == idf.IDF_ETIMEOUT
    assert "wait" in W.last_error()
    with pytest.raises(idf.IdfError) as e:
        W.query(*RECT)
    assert e.value.status == idf.IDF_EINTERNAL
    W.close()
    # the context is intact: a new world reproduces the result bit for bit
    W2 = idf.World(0, st, wts, precision="tf32")
    assert np.array_equal(W2.query(*RECT), good)
    W2.close()


def test_bounds_check_flag_is_reported_and_cleared(idf):
    st = synth.small_hier_stack(steps=2)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    W = idf.World(0, st, wts, precision="fp32")
    good = W.query(*RECT).copy()
    W.cache_clear()
    W.debug_set_status(1, 1)
    with pytest.raises(idf.IdfError) as e:
        W.query(*RECT)
    assert e.value.status == idf.IDF_EDEVICE_CHECK
    # not poisoning: the flag was cleared and the next query is correct
    W.cache_clear()
    assert np.array_equal(W.query(*RECT), good)
    W.close()


def test_injection_rejects_unknown_word(idf):
    st = synth.config1_stack(test_denoiser=1)
    W = idf.World(0, st, None)
    with pytest.raises(idf.IdfError) as e:
        W.debug_set_status(2, 1)
    assert e.value.status == idf.IDF_EINVAL
    W.close()
