"""The learned student trained by the library's own forward and backward
kernels: loss and gradients against the FP64 oracle (torch autograd, pinned
by finite differences in test_oracle_student.py), AdamW against its formula,
and training that lowers the loss."""
import numpy as np
import pytest

import synth
from oracle import student as OST
from oracle import unet as OU

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def idf():
    import paper_2512_08309_gb300 as m
    m.lib()
    return m


def _w(lv, seed):
    return synth.weights([s for _, s in OU.param_shapes(lv)], seed, 0)


def _batch(n, H, seed):
    rng = np.random.default_rng(seed)
    x = (rng.standard_normal((n, H, H)) * 3.0).astype(np.float32)
    t = (rng.standard_normal((n, H, H)) * 0.3).astype(np.float32)
    return x, t


@pytest.mark.parametrize("lv,n,sigma", [
    (synth.level(levels=2, channels=(8, 8), in_ch=1, out_ch=1, window=16, gn_groups=4), 3, 0.8),
    (synth.level(levels=3, channels=(16, 32, 32), in_ch=1, out_ch=1, window=32, gn_groups=4), 2, 80.0),
])
def test_loss_and_gradient_match_oracle(idf, lv, n, sigma):
    w = _w(lv, 1)
    x, t = _batch(n, lv["window"], 2)
    S = idf.Student(lv, w, max_batch=4)
    loss = S.loss_grad(torch.from_numpy(x).cuda().data_ptr(), torch.from_numpy(t).cuda().data_ptr(), n, sigma)
    g = S.grads().astype(np.float64)
    S.close()
    ref_loss, ref_g = OST.loss_and_grad(lv, w.astype(np.float64), x, t, sigma)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert np.max(np.abs(g - ref_g)) <= 1e-4 * np.max(np.abs(ref_g))


def test_student_width_gradient_matches_oracle(idf):
    # the student of the distillation (32/64/128/128 channels, 128x128 windows)
    lv = synth.student_level()
    w = _w(lv, 3)
    x, t = _batch(2, 128, 4)
    x *= 80.0 / 3.0
    S = idf.Student(lv, w, max_batch=2)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss = S.loss_grad(xd.data_ptr(), td.data_ptr(), 2, 80.0)
    g = S.grads().astype(np.float64)
    S.close()
    ref_loss, ref_g = OST.loss_and_grad(lv, w.astype(np.float64), x, t, 80.0)
    d = g - ref_g
    print(f"loss {loss:.6e} ref {ref_loss:.6e}; grad max err {np.max(np.abs(d)) / np.max(np.abs(ref_g)):.3e} of max")
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert np.max(np.abs(d)) <= 1e-3 * np.max(np.abs(ref_g))


def test_adamw_step_matches_formula(idf):
    lv = synth.level(levels=2, channels=(8, 8), in_ch=1, out_ch=1, window=16, gn_groups=4)
    w = _w(lv, 5)
    x, t = _batch(2, 16, 6)
    S = idf.Student(lv, w, max_batch=2)
    S.loss_grad(torch.from_numpy(x).cuda().data_ptr(), torch.from_numpy(t).cuda().data_ptr(), 2, 1.0)
    g = S.grads().astype(np.float64)
    S.adamw(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01)
    w1 = S.weights().astype(np.float64)
    assert np.all(S.grads() == 0.0)
    S.close()
    ref, _, _ = OST.adamw(w.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-3, wd=0.01)
    assert np.max(np.abs(w1 - ref)) <= 1e-6


def test_training_lowers_the_loss(idf):
    lv = synth.level(levels=3, channels=(16, 32, 32), in_ch=1, out_ch=1, window=32, gn_groups=4)
    w = _w(lv, 7)
    x, t = _batch(8, 32, 8)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    S = idf.Student(lv, w, max_batch=8)
    losses = []
    for _ in range(60):
        losses.append(S.loss_grad(xd.data_ptr(), td.data_ptr(), 8, 0.35))
        S.adamw(lr=2e-3)
    S.close()
    print("loss", losses[0], "->", losses[-1])
    assert losses[-1] < 0.5 * losses[0]
