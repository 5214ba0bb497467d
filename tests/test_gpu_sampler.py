"""GPU parity of the sampling path (noise, scheduler, blend, cache, decode)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import noise as ON
from oracle import kappa as OK
from oracle import laplacian as OL
from oracle import sampler as OS
from oracle import unet as OU

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def idf():
    import paper_2512_08309_gb300 as m
    m.lib()
    assert torch.cuda.is_available()
    return m


def weights_for(st, seed=0):
    return [synth.weights([s for _, s in OU.param_shapes(lv)], seed, li) if not lv["test_denoiser"] else None
            for li, lv in enumerate(st["level"])]


# --------------------------------------------------------------------- noise

@pytest.mark.parametrize("seed,level,step,x0,y0,w,h", [
    (0, 0, 0, 0, 0, 257, 131),
    (0xDEADBEEFCAFEF00D, 1, 19, -1000, -37, 300, 64),
    (7, 3, 2, (1 << 31) - 100, -(1 << 31) - 50, 200, 100),     # counter wrap at 2^32
    (123, 0, 5, -(1 << 40), (1 << 40) - 8, 64, 16),
])
def test_noise_bit_exact(idf, seed, level, step, x0, y0, w, h):
    out = torch.empty((h, w + 3), dtype=torch.float32, device="cuda")
    idf.noise_fill(seed, level, step, x0, y0, w, h, out.data_ptr(), w + 3)
    torch.cuda.synchronize()
    got = out[:, :w].cpu().numpy()
    ref = ON.normal_region(seed, level, step, x0, y0, w, h)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


# --------------------------------------------------------------- scheduler

def test_debug_cone_matches_oracle_recursion(idf):
    st = synth.config1_stack(test_denoiser=1)
    W = idf.World(0, st)
    lv = st["level"][0]
    for rect in [(0, 0, 64, 64), (-37, 5, 20, 50), (16, 16, 1, 1)]:
        x0, y0, w, h = rect
        rects = OS.cone_rects(OS.Level(0, lv, 0), y0, x0, h, w)
        for step in range(lv["steps"]):
            ry0, rx0, rh, rw = rects[step + 1]
            # windows of step k are kappa of the region of J_{k+1}; the library
            # works on whole tiles, so compare against kappa of the tile-aligned region
            s = lv["stride"]
            ty0, tx0 = ry0 // s, rx0 // s
            ty1, tx1 = (ry0 + rh - 1) // s, (rx0 + rw - 1) // s
            ref = OK.kappa(ty0 * s, tx0 * s, (ty1 - ty0 + 1) * s, (tx1 - tx0 + 1) * s, lv["window"], s)
            assert W.debug_cone(x0, y0, w, h, 0, step) == ref
    W.close()


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("td", [1, 2, 3])
def test_test_denoisers_match_oracle(idf, td):
    st = synth.config1_stack(test_denoiser=td)
    W = idf.World(11, st)
    for rect in [(0, 0, 64, 64), (-45, 17, 37, 29)]:
        x0, y0, w, h = rect
        got = W.query(x0, y0, w, h).astype(np.float64)
        ref = OS.World(11, st, None).model(y0, x0, h, w)
        assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))
    W.close()


def test_test_denoiser_full_geometry_2level(idf):
    # the 2-level stack geometry of the 4096^2 workload (128 windows at stride
    # 64, 20 steps, conditioning, Laplacian decode) with closed-form denoisers:
    # sampled pixels against the oracle's lazy world
    st = synth.config2_stack(test_denoiser=3)
    W = idf.World(5, st)
    x0, y0, w, h = -300, 1200, 700, 300
    got = W.query(x0, y0, w, h, kind=idf.IDF_OUT_METRES)
    oracle = OS.World(5, st, None)
    rng = np.random.default_rng(0)
    for _ in range(3):
        r, c = int(rng.integers(0, h)), int(rng.integers(0, w))
        ref = oracle.metres(y0 + r, x0 + c, 1, 1)[0, 0]
        assert abs(got[r, c] - ref) <= 1e-4 * max(1.0, abs(ref))
    gm = W.query(x0, y0, 64, 64)
    om = oracle.model(y0, x0, 64, 64)
    assert np.max(np.abs(gm - om)) <= 2e-5 * np.max(np.abs(om))
    W.close()


# --------------------------------------------------------------- UNet path

def test_config1_fp32_query_matches_oracle(idf):
    st = synth.config1_stack()
    wts = weights_for(st)
    W = idf.World(0, st, wts, precision="fp32")
    got = W.query(0, 0, 64, 64).astype(np.float64)
    ref = OS.World(0, st, wts).model(0, 0, 64, 64)
    sig = ref.std()
    err = np.max(np.abs(got - ref))
    assert err <= 1e-4 * sig, (err, sig)
    stats = W.stats()
    assert stats["levels"][0]["windows_evaluated"] == 276
    W.close()


def test_small_hierarchy_matches_oracle(idf):
    st = synth.small_hier_stack(steps=2, window=16, stride=8, coarse_channels=(8, 8), fine_channels=(8, 16))
    wts = weights_for(st)
    W = idf.World(3, st, wts, precision="fp32")
    oracle = OS.World(3, st, wts)
    got = W.query(-20, 3, 24, 20).astype(np.float64)
    ref = oracle.model(3, -20, 20, 24)
    assert np.max(np.abs(got - ref)) <= 1e-4 * ref.std()
    gm = W.query(-20, 3, 24, 20, kind=idf.IDF_OUT_METRES).astype(np.float64)
    rm = oracle.metres(3, -20, 20, 24)
    # metres error, first order 2|v| dv: compare in signed-sqrt units
    gv = np.sign(gm) * np.sqrt(np.abs(gm))
    rv = np.sign(rm) * np.sqrt(np.abs(rm))
    assert np.max(np.abs(gv - rv)) <= 2e-4 * rv.std()
    W.close()


# ------------------------------------------------- order / cache / batching

def test_order_cache_and_batch_independence_bitwise(idf):
    st = synth.with_steps(synth.config1_stack(), 3)
    wts = weights_for(st)
    A = idf.World(9, st, wts)
    a1 = A.query(0, 0, 96, 80)
    a2 = A.query(40, 50, 70, 90)
    B = idf.World(9, st, wts, cache_bytes=1 << 22)   # small cache: evictions between queries
    b2 = B.query(40, 50, 70, 90)
    b1 = B.query(0, 0, 96, 80)
    assert np.array_equal(a1, b1) and np.array_equal(a2, b2)
    assert np.array_equal(a1[50:80, 40:96], a2[0:30, 0:56])
    B.cache_clear()
    assert np.array_equal(B.query(0, 0, 96, 80), a1)
    C = idf.World(9, st, wts)
    o1 = torch.zeros((80, 96), device="cuda")
    o2 = torch.zeros((90, 70), device="cuda")
    C.query_batch([(0, 0, 96, 80, o1.data_ptr(), 96), (40, 50, 70, 90, o2.data_ptr(), 70)])
    torch.cuda.synchronize()
    assert np.array_equal(o1.cpu().numpy(), a1) and np.array_equal(o2.cpu().numpy(), a2)
    for w in (A, B, C):
        w.close()


def test_invalid_arguments(idf):
    st = synth.config1_stack(test_denoiser=1)
    W = idf.World(0, st)
    with pytest.raises(idf.IdfError) as e:
        W.query(0, 0, 0, 5)
    assert e.value.status == idf.IDF_EINVAL
    with pytest.raises(idf.IdfError) as e:
        W.query(0, 0, 8, 8, kind=idf.IDF_OUT_METRES)
    assert e.value.status == idf.IDF_EINVAL
    # the world stays usable after argument errors
    assert W.query(0, 0, 8, 8).shape == (8, 8)
    bad = synth.config1_stack()
    with pytest.raises(idf.IdfError) as e:
        idf.World(0, bad, [np.zeros(10, np.float32)])
    assert e.value.status == idf.IDF_EMODEL
    W.close()


def test_cache_too_small_is_enomem_and_recoverable(idf):
    st = synth.config1_stack(test_denoiser=2)
    W = idf.World(0, st, cache_bytes=16 * 16 * 4 * 100)   # 100 tiles: an 8x8 query needs 84
    with pytest.raises(idf.IdfError) as e:
        W.query(0, 0, 64, 64)
    assert e.value.status == idf.IDF_ENOMEM
    W.cache_clear()
    out = W.query(0, 0, 8, 8)
    ref = OS.World(0, st, None).model(0, 0, 8, 8)
    assert np.max(np.abs(out - ref)) <= 2e-6 * np.max(np.abs(ref))
    W.close()


# ------------------------------------------------------------------ decode

def test_laplacian_decode_matches_oracle(idf):
    st = synth.config2_stack()
    x0, y0, w, h = -517, 2048, 700, 333
    Lr, Hr = idf.laplacian_halo(st, x0, y0, w, h)
    rng = np.random.default_rng(1)
    Lb = rng.standard_normal((Lr[3], Lr[2])).astype(np.float32)
    Hb = rng.standard_normal((Hr[3], Hr[2])).astype(np.float32)
    Ld, Hd = torch.from_numpy(Lb).cuda(), torch.from_numpy(Hb).cuda()
    out = torch.empty((h, w), device="cuda")
    idf.laplacian_decode(st, Ld.data_ptr(), Lr, Lr[2], Hd.data_ptr(), Hr, Hr[2], x0, y0, w, h, out.data_ptr(), w)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)

    def Lf(cy0, cx0, ch, cw):
        return Lb[cy0 - Lr[1]:cy0 - Lr[1] + ch, cx0 - Lr[0]:cx0 - Lr[0] + cw]

    def Hf(fy0, fx0, fh, fw):
        return Hb[fy0 - Hr[1]:fy0 - Hr[1] + fh, fx0 - Hr[0]:fx0 - Hr[0] + fw]

    ref = OL.decode_metres(Lf, Hf, y0, x0, h, w)
    # float32 arithmetic on values up to ~ (4 * 50)^2 metres
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
    # a band that does not cover the halo is rejected
    with pytest.raises(idf.IdfError):
        idf.laplacian_decode(st, Ld.data_ptr(), (Lr[0] + 1, Lr[1], Lr[2] - 1, Lr[3]), Lr[2], Hd.data_ptr(), Hr,
                             Hr[2], x0, y0, w, h, out.data_ptr(), w)


# ------------------------------------------------------ degenerate layouts

@pytest.mark.parametrize("window,stride,steps", [
    (16, 16, 3),   # window = stride: independent tiles (no overlap, Sec. 6 baseline)
    (48, 16, 2),   # three windows per tile and axis
    (32, 16, 1),   # a single blended step
])
def test_layouts_match_oracle(idf, window, stride, steps):
    lv = synth.level(window=window, stride=stride, steps=steps, test_denoiser=3)
    st = synth.stack([lv])
    W = idf.World(2, st)
    x0, y0, w, h = -37, 21, 45, 33
    got = W.query(x0, y0, w, h).astype(np.float64)
    W.close()
    ref = OS.World(2, st, None).model(y0, x0, h, w)
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_extreme_coordinates(idf):
    st = synth.config1_stack(test_denoiser=2)
    W = idf.World(0, st)
    # tile indices near the int32 limit still work and agree with the oracle
    x0 = (1 << 31) * 16 - 16 * 40
    got = W.query(x0, -x0, 16, 8).astype(np.float64)
    ref = OS.World(0, st, None).model(-x0, x0, 8, 16)
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))
    # beyond it the request is refused, and the world stays usable
    with pytest.raises(idf.IdfError) as e:
        W.query((1 << 40) - 64, 0, 8, 8)
    assert e.value.status == idf.IDF_EINVAL
    with pytest.raises(idf.IdfError) as e:
        W.query_device(0, 0, 1 << 16, (1 << 15) + 1, 0, 1 << 16)
    assert e.value.status == idf.IDF_EINVAL
    assert W.query(0, 0, 4, 4).shape == (4, 4)
    W.close()
