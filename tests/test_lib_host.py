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
    assert len(syms) == 33
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


@pytest.mark.parametrize("case", ["two_level_with_fixture", "fixture_without_laplacian",
                                  "single_level_laplacian_without_fixture", "fixture_with_conditioned_level"])
def test_world_create_rejects_invalid_low_band_setups(case):
    # argument validation runs before any device call, so a bad stack is
    # refused with IDF_EINVAL even without a GPU
    import numpy as np
    idf = _lib()
    fx = np.zeros((8, 8), dtype=np.float32)
    if case == "two_level_with_fixture":
        st = synth.small_hier_stack(test_denoiser=1)
        st["low_band_fixture"] = fx
    elif case == "fixture_without_laplacian":
        st = synth.config4_stack(fx, test_denoiser=1)
        st["laplacian"] = 0
    elif case == "single_level_laplacian_without_fixture":
        st = synth.config4_stack(fx, test_denoiser=1)
        st.pop("low_band_fixture")
    else:
        st = synth.config4_stack(fx, test_denoiser=1)
        st["level"][0]["in_ch"] = 2
    with pytest.raises(idf.IdfError) as e:
        idf.World(0, st, [None] * len(st["level"]))
    assert e.value.status == idf.IDF_EINVAL


def test_world_create_accepts_a_single_level_low_band_setup():
    # the valid form passes validation; without a GPU it stops at the device
    # call (IDF_ECUDA), with one it creates the world
    import numpy as np
    idf = _lib()
    st = synth.config4_stack(np.zeros((8, 8), dtype=np.float32), test_denoiser=1)
    try:
        idf.World(0, st, [None]).close()
    except idf.IdfError as e:
        assert e.status == idf.IDF_ECUDA


def test_missing_library_fails_loudly(tmp_path):
    # with libidf absent the binding raises on its first call: there is no
    # other implementation behind it (a subprocess, so that the library this
    # process has loaded stays untouched)
    import subprocess
    import sys
    code = ("import paper_2512_08309_gb300 as idf, synth\n"
            f"idf.LIB_PATH = {str(tmp_path / 'absent' / 'libidf.so')!r}\n"
            "for call in (lambda: idf.lib(), lambda: idf.World(0, synth.config2_stack(), [None, None])):\n"
            "    try:\n"
            "        call()\n"
            "    except RuntimeError as e:\n"
            "        assert 'not built' in str(e), e\n"
            "    else:\n"
            "        raise SystemExit('no error without the library')\n")
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
