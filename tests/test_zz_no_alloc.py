"""The allocation-free Laplacian decode.

Some callers cannot allocate device memory when they call the library (a
plugin inside an engine that owns all device memory through its own pool, a
frame loop that cannot take an allocation's latency).  For them
idf_laplacian_decode_noalloc runs the decode with a fixed scratch array in
the library's device image.  This file checks, through the C ABI, that it
returns what idf_laplacian_decode returns, on two calls in a row (the second
reuses the array the first left behind), and that a query too large for the
fixed array is refused.  It is named so that pytest collects it last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _bands(idf, st, x0, y0, w, h, seed):
    Lr, Hr = idf.laplacian_halo(st, x0, y0, w, h)
    rng = np.random.default_rng(seed)
    L = torch.from_numpy(rng.standard_normal((Lr[3], Lr[2])).astype(np.float32)).cuda()
    H = torch.from_numpy(rng.standard_normal((Hr[3], Hr[2])).astype(np.float32)).cuda()
    return Lr, Hr, L, H


def test_noalloc_decode_matches_allocating_decode_twice():
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st = synth.config2_stack()
    for call, (x0, y0, w, h) in enumerate([(-517, 2048, 700, 333), (4096, -77, 256, 1024)]):
        Lr, Hr, L, H = _bands(idf, st, x0, y0, w, h, seed=call)
        ref = torch.empty((h, w), device="cuda")
        got = torch.full((h, w), float("nan"), device="cuda")
        idf.laplacian_decode(st, L.data_ptr(), Lr, Lr[2], H.data_ptr(), Hr, Hr[2], x0, y0, w, h,
                             ref.data_ptr(), w)
        idf.laplacian_decode_noalloc(st, L.data_ptr(), Lr, Lr[2], H.data_ptr(), Hr, Hr[2], x0, y0, w, h,
                                     got.data_ptr(), w)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy().astype(np.float64), got.cpu().numpy().astype(np.float64)
        # the tolerance of the decode parity test (float32 arithmetic)
        assert np.all(np.isfinite(g))
        assert np.max(np.abs(g - r)) <= 1e-5 * np.max(np.abs(r))


def test_noalloc_decode_rejects_queries_beyond_its_scratch():
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st = synth.config2_stack()
    x0, y0, w, h = 0, 0, 8192, 8192
    Lr, Hr = idf.laplacian_halo(st, x0, y0, w, h)
    # buffers of the true sizes, so that nothing could be read out of bounds
    L = torch.zeros((Lr[3], Lr[2]), device="cuda")
    H = torch.zeros((Hr[3], Hr[2]), device="cuda")
    out = torch.zeros((h, w), device="cuda")
    with pytest.raises(idf.IdfError) as e:
        idf.laplacian_decode_noalloc(st, L.data_ptr(), Lr, Lr[2], H.data_ptr(), Hr, Hr[2], x0, y0, w, h,
                                     out.data_ptr(), w)
    assert e.value.status == idf.IDF_EINVAL


def test_noalloc_decode_matches_the_oracle_decode():
    # directly against the FP64 oracle's decode of the same bands (its
    # device-computed blur taps may differ from the host's in the last bit)
    import paper_2512_08309_gb300 as idf
    from oracle import laplacian as OL
    idf.lib()
    st = synth.config2_stack()
    x0, y0, w, h = -301, 77, 200, 150
    Lr, Hr, L, H = _bands(idf, st, x0, y0, w, h, seed=7)
    got = torch.full((h, w), float("nan"), device="cuda")
    idf.laplacian_decode_noalloc(st, L.data_ptr(), Lr, Lr[2], H.data_ptr(), Hr, Hr[2], x0, y0, w, h,
                                 got.data_ptr(), w)
    torch.cuda.synchronize()
    Ln, Hn = L.cpu().numpy().astype(np.float64), H.cpu().numpy().astype(np.float64)

    def lfun(cy0, cx0, ch, cw):
        return Ln[cy0 - Lr[1]:cy0 - Lr[1] + ch, cx0 - Lr[0]:cx0 - Lr[0] + cw]

    def hfun(yy0, xx0, hh, ww):
        return Hn[yy0 - Hr[1]:yy0 - Hr[1] + hh, xx0 - Hr[0]:xx0 - Hr[0] + ww]

    ref = OL.decode_metres(lfun, hfun, y0, x0, h, w, factor=st["lap_factor"], blur_sigma=st["lap_blur_sigma"],
                           radius=st["lap_radius"], low_mu=st["low_mu"], low_scale=st["low_scale"],
                           res_scale=st["res_scale"])
    g = got.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - ref)) <= 1e-5 * np.max(np.abs(ref))
