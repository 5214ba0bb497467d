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
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()   # keep the buffers alive
    loss = S.loss_grad(xd.data_ptr(), td.data_ptr(), n, sigma)
    g = S.grads().astype(np.float64)
    S.close()
    ref_loss, ref_g = OST.loss_and_grad(lv, w.astype(np.float64), x, t, sigma)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    assert np.max(np.abs(g - ref_g)) <= 1e-4 * np.max(np.abs(ref_g))


def test_side_channel_loss_and_gradient_match_oracle(idf):
    # in_ch = 4: the noisy state in channel 0, three side fields unscaled
    lv = synth.level(levels=2, channels=(8, 16), in_ch=4, out_ch=1, window=16, gn_groups=4)
    w = _w(lv, 5)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((3, 4, 16, 16)).astype(np.float32)
    x[:, 0] *= 80.0
    t = (rng.standard_normal((3, 16, 16)) * 0.3).astype(np.float32)
    S = idf.Student(lv, w, max_batch=4)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    loss = S.loss_grad(xd.data_ptr(), td.data_ptr(), 3, 80.0)
    g = S.grads().astype(np.float64)
    S.close()
    ref_loss, ref_g = OST.loss_and_grad(lv, w.astype(np.float64), x, t, 80.0)
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
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    S.loss_grad(xd.data_ptr(), td.data_ptr(), 2, 1.0)
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


def test_distillation_gain_over_untrained_student(idf):
    # Pairs from the plain 16-channel sampler (targets: 128 x 128 crops of its
    # output; inputs: its own initial noise sigma_0 N(seed, 0, 0, .) there);
    # training must lower the held-out loss below the untrained student's.
    c1 = synth.config1_stack()
    c1w = [synth.weights(idf.param_shapes(lv), 0, i) for i, lv in enumerate(c1["level"])]
    plain = idf.World(0, c1, c1w, precision="fp32")
    H, side = 128, 512
    T, N0 = [], []
    for q in range(3):
        x0, y0 = (q * 7 + 1) * (1 << 20), (q * 13 + 5) * (1 << 19)
        big = plain.query(x0, y0, side, side)
        for a in range(side // H):
            for b in range(side // H):
                T.append(big[a * H:(a + 1) * H, b * H:(b + 1) * H])
                n0 = torch.empty((H, H), device="cuda")
                idf.noise_fill(0, 0, 0, x0 + b * H, y0 + a * H, H, H, n0.data_ptr(), H)
                N0.append(n0)
    plain.close()
    T = torch.from_numpy(np.stack(T)).cuda()
    X = 80.0 * torch.stack(N0)
    tr, ho = slice(0, 40), slice(40, 48)
    lv = synth.student_level()
    S = idf.Student(lv, synth.weights(idf.param_shapes(lv), 0, 0), max_batch=8)

    def held_out():
        x, t = X[ho].contiguous(), T[ho].contiguous()
        v = S.loss_grad(x.data_ptr(), t.data_ptr(), 8, 80.0)
        S.zero_grad()
        return v

    before = held_out()
    for it in range(25):
        i = (it * 8) % 40
        x, t = X[i:i + 8].contiguous(), T[i:i + 8].contiguous()
        S.loss_grad(x.data_ptr(), t.data_ptr(), 8, 80.0)
        S.adamw(lr=1e-3)
    after = held_out()
    S.close()
    print(f"held-out loss {before:.4e} -> {after:.4e}")
    assert after < 0.9 * before


def test_autograd_function_against_finite_differences(idf):
    # the loss as a torch.autograd.Function over the library's forward and
    # backward kernels: its gradient against central finite differences of
    # the same loss along random directions, and a torch optimiser driving
    # the library's training step
    from paper_2512_08309_gb300.autograd import student_loss
    lv = synth.level(levels=2, channels=(8, 8), in_ch=1, out_ch=1, window=16, gn_groups=4)
    w0 = _w(lv, 5)
    x, t = _batch(3, 16, 6)
    S = idf.Student(lv, w0, max_batch=4)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    w = torch.tensor(w0, requires_grad=True)
    loss = student_loss(w, xd, td, 0.8, S)
    loss.backward()
    g = w.grad.detach().numpy().astype(np.float64)
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.standard_normal(w0.size)
        v /= np.linalg.norm(v)
        h = 1e-2
        lp = float(student_loss(torch.tensor((w0 + h * v).astype(np.float32)), xd, td, 0.8, S))
        lm = float(student_loss(torch.tensor((w0 - h * v).astype(np.float32)), xd, td, 0.8, S))
        fd = (lp - lm) / (2 * h)
        an = float(g @ v)
        print(f"directional derivative: autograd {an:.6e}, finite differences {fd:.6e}")
        assert abs(fd - an) <= 2e-2 * abs(an) + 1e-6
    # a torch optimiser over the Function lowers the loss
    w = torch.tensor(w0, requires_grad=True)
    opt = torch.optim.AdamW([w], lr=2e-3)
    first = None
    for _ in range(20):
        opt.zero_grad()
        l = student_loss(w, xd, td, 0.8, S)
        l.backward()
        opt.step()
        first = float(l) if first is None else first
    assert float(student_loss(w, xd, td, 0.8, S)) < first
    S.close()
