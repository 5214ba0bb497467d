"""Student denoiser training (oracle): loss, gradients and AdamW, FP64.

Test infrastructure (see the package header).

The paper distils its networks into few-step continuous-time consistency
models (Sec. 5.4, App. F "Consistency Distillation"); the learned
part is a plain few-step student trained by regression, read as follows:

* network S: the same ResBlock UNet as ``oracle.unet`` (its layer reading and
  parameter order), here written with torch operations in float64 so that
  torch.autograd gives exact gradients;
* preconditioning as for every denoiser: D(x; sigma) = c_skip x + c_out
  S(c_in x); with side inputs (in_ch > 1: x of shape (B, in_ch, H, W))
  channel 0 is the noisy state and the others are given to S as they are,
  D = c_skip x_0 + c_out S([c_in x_0, x_1, ...]);
* loss of a batch at one sigma: mean over pixels of (D(x; sigma) - t)^2,
  where t is the plain sampler's output over the window and x the noisy
  input (pure noise sigma_0 N at sigma = 80, or t + sigma_mid N at
  sigma_mid = 0.35, the paper's intermediate consistency sigma of the core
  model, Table "Hyperparameters");
* AdamW (Loshchilov and Hutter, "Decoupled weight decay regularization"):
  m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, mh = m / (1 - b1^t),
  vh = v / (1 - b2^t), w = w - lr (mh / (sqrt(vh) + eps) + wd w).

Pins: the float64 torch forward equals ``oracle.unet.forward``; gradients
equal central finite differences (tests/test_oracle_student.py); one AdamW
step is checked against its formula evaluated by hand for scalars.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as TF

from . import schedule as S_
from . import unet as U_


def _params(lv: dict, flat: np.ndarray, requires_grad: bool = True):
    shapes = U_.param_shapes(lv)
    flat = torch.as_tensor(np.asarray(flat, dtype=np.float64))
    out, o = {}, 0
    for name, s in shapes:
        k = int(np.prod(s))
        t = flat[o:o + k].reshape(s).clone()
        t.requires_grad_(requires_grad)
        out[name] = t
        o += k
    return out


def forward_torch(lv: dict, p: dict, x: torch.Tensor) -> torch.Tensor:
    """F(x), x (B, in_ch, H, W) float64, with the layer reading of oracle.unet."""
    G = int(lv["gn_groups"])

    def gn(h):
        return TF.group_norm(h, G, eps=U_.GN_EPS)

    def conv(h, w):
        return TF.conv2d(h, w, padding=w.shape[-1] // 2)

    def rb(h, name):
        a = conv(TF.silu(gn(h)), p[name + ".conv1"])
        a = conv(TF.silu(gn(a)), p[name + ".conv2"])
        return a + (conv(h, p[name + ".skip"]) if name + ".skip" in p else h)

    L = int(lv["levels"])
    h = conv(x, p["in_conv"])
    skips = []
    for l in range(L):
        h = rb(h, f"enc{l}")
        skips.append(h)
        if l < L - 1:
            h = TF.avg_pool2d(h, 2)
    if int(lv.get("attn_at_bottom", 0)):
        raise ValueError("the student has no attention block")
    h = rb(h, "mid")
    for l in range(L - 2, -1, -1):
        h = torch.cat([h.repeat_interleave(2, dim=2).repeat_interleave(2, dim=3), skips[l]], dim=1)
        h = rb(h, f"dec{l}")
    return conv(TF.silu(gn(h)), p["out_conv"])


def _denoise(lv: dict, p: dict, x: np.ndarray, sigma: float):
    """D(x; sigma), x (B, H, W) or (B, in_ch, H, W) with side channels."""
    c_skip, c_out, c_in = S_.edm_coeffs(float(sigma), float(lv["sigma_data"]))
    xt = torch.as_tensor(np.asarray(x, dtype=np.float64))
    if xt.dim() == 3:
        xt = xt[:, None]
    x0 = xt[:, :1]
    xin = torch.cat([c_in * x0, xt[:, 1:]], dim=1)
    return c_skip * x0 + c_out * forward_torch(lv, p, xin)


def loss_and_grad(lv: dict, flat: np.ndarray, x: np.ndarray, target: np.ndarray, sigma: float):
    """Loss mean((D(x; sigma) - t)^2) and its gradient w.r.t. the flat weights
    (declaration order).  x: (B, H, W), or (B, in_ch, H, W) with side
    channels; target: (B, H, W)."""
    p = _params(lv, flat, True)
    tt = torch.as_tensor(np.asarray(target, dtype=np.float64))[:, None]
    D = _denoise(lv, p, x, sigma)
    loss = ((D - tt) ** 2).mean()
    loss.backward()
    g = torch.cat([p[n].grad.reshape(-1) for n, _ in U_.param_shapes(lv)])
    return float(loss.detach()), g.numpy()


def loss_only(lv: dict, flat: np.ndarray, x: np.ndarray, target: np.ndarray, sigma: float) -> float:
    with torch.no_grad():
        p = _params(lv, flat, False)
        tt = torch.as_tensor(np.asarray(target, dtype=np.float64))[:, None]
        D = _denoise(lv, p, x, sigma)
        return float(((D - tt) ** 2).mean())


def adamw(w, g, m, v, t, lr=2e-4, b1=0.9, b2=0.999, eps=1e-8, wd=0.01):
    """One AdamW step (t counts from 1); returns new (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    w = w - lr * (mh / (np.sqrt(vh) + eps) + wd * w)
    return w, m, v
