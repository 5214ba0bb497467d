"""Host-side checks of libidf that need no GPU: the library loads, exports
every symbol include/idf.h declares, and its host logic (parameter layout,
decode halo) agrees with the oracle."""
import os
import re

import pytest

import synth
from oracle import laplacian as OL
from oracle import unet as OU

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import paper_2512_08309_gb300 as idf
    if not os.path.exists(idf.LIB_PATH):
        from paper_2512_08309_gb300 import build
        build.build()
    return idf


def header_symbols():
    src = open(os.path.join(ROOT, "include", "idf.h")).read()
    return sorted(set(re.findall(r"^(?:idf_status|void|const char\*)\s+(idf_\w+)\(", src, re.M)))


def test_header_symbols_exported():
    idf = _lib()
    L = idf.lib()
    syms = header_symbols()
    assert len(syms) == 23
    for s in syms:
        assert hasattr(L, s), s
    assert sorted(idf.EXPORTS) == syms


@pytest.mark.parametrize("lv", [
    synth.config1_stack()["level"][0],
    synth.config2_stack()["level"][0],
    synth.config2_stack()["level"][1],
    synth.small_hier_stack()["level"][1],
])
def test_param_shapes_match_oracle(lv):
    idf = _lib()
    assert idf.param_shapes(lv) == [tuple(s) for _, s in OU.param_shapes(lv)]


@pytest.mark.parametrize("rect", [(0, 0, 64, 64), (-77, 301, 23, 57), (5, -9, 1, 1), (4095, -4096, 8, 9)])
def test_decode_halo_covers_oracle_reads(rect):
    idf = _lib()
    st = synth.config2_stack()
    x0, y0, w, h = rect
    Lr, Hr = idf.laplacian_halo(st, x0, y0, w, h)
    # the oracle's decode reads exactly these rects (rows from y, cols from x)
    f, R = 8, 15
    qy0, qy1 = OL.up_range(y0, h, f)
    qx0, qx1 = OL.up_range(x0, w, f)
    py0, px0 = f * (qy0 - R), f * (qx0 - R)
    ph, pw = f * (qy1 - qy0 + 1 + 2 * R), f * (qx1 - qx0 + 1 + 2 * R)
    ly0, ly1 = OL.up_range(py0, ph, f)
    lx0, lx1 = OL.up_range(px0, pw, f)
    assert Hr == (px0, py0, pw, ph)
    assert Lr == (lx0, ly0, lx1 - lx0 + 1, ly1 - ly0 + 1)
