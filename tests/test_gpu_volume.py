"""InfiniteDiffusion on Z^3 (voxel volumes) against the FP64 oracle: the
closed-form test denoisers, the small 3-D network, the cone's window count,
and query-order and cache-size independence."""
import numpy as np
import pytest

import synth
from oracle import volume as OV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def idf():
    import paper_2512_08309_gb300 as m
    m.lib()
    return m


@pytest.mark.parametrize("td", [1, 2, 3])
def test_volume_test_denoisers(idf, td):
    desc = synth.volume_desc(test_denoiser=td)
    box = (-13, 9, -5, 9, 6, 7)          # x0, y0, z0, w, h, d
    V = idf.Volume(3, desc)
    got = V.query(*box).astype(np.float64)
    V.close()
    ref = OV.VolumeLevel(3, desc).final(box[2], box[1], box[0], box[5], box[4], box[3])
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_volume_network_against_oracle(idf):
    desc = synth.volume_desc(steps=2)
    w = synth.volume_weights(desc)
    box = (-8, 0, 8, 16, 12, 8)
    V = idf.Volume(0, desc, w)
    got = V.query(*box).astype(np.float64)
    st = V.stats()
    V.close()
    lz = OV.VolumeLevel(0, desc, w)
    ref = lz.final(box[2], box[1], box[0], box[5], box[4], box[3])
    err = float(np.max(np.abs(got - ref)) / ref.std())
    print(f"3-D network: max {err:.3e} sigma_out, {st['windows_evaluated']} windows")
    assert err <= 1e-4
    assert st["windows_evaluated"] == lz.phi_calls


def test_volume_cone_count_order_and_cache(idf):
    desc = synth.volume_desc(test_denoiser=2)
    V = idf.Volume(1, desc)
    a = V.query(0, 0, 0, 16, 16, 16)     # 2 x 2 x 2 tiles, cold
    assert V.stats()["windows_evaluated"] == sum((2 + 2 * k + 1) ** 3 for k in range(3))
    b = V.query(8, 8, 8, 16, 16, 16)     # overlaps: partly cached
    V.close()
    W = idf.Volume(1, desc, cache_bytes=64 * 8 ** 3 * 4 * 8)   # small cache: evictions
    b2 = W.query(8, 8, 8, 16, 16, 16)
    a2 = W.query(0, 0, 0, 16, 16, 16)
    W.close()
    assert np.array_equal(a, a2) and np.array_equal(b, b2)
    assert np.array_equal(a[8:, 8:, 8:], b[:8, :8, :8])
