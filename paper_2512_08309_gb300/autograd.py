"""torch.autograd binding of the student's loss (argument marshalling only).

``StudentLoss.apply(weights, x, target, sigma, student)`` evaluates the
preconditioned denoising loss mean((D(x; sigma) - target)^2) of the library
student on a batch of windows (x, target: CUDA float32 (n, H, H)) and, in
backward, returns its gradient with respect to ``weights`` (a float32 tensor
of the parameter count, declaration order).  Both passes run in the
library's own forward and backward kernels (idf_student_loss_grad); this
module only moves weights and gradients between torch tensors and the
student, so autograd, optimisers and gradient checks in torch drive the
library's training path.
"""
from __future__ import annotations

import numpy as np


def _torch():
    import torch
    return torch


def _make():
    torch = _torch()

    class StudentLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, weights, x, target, sigma, student):
            w = weights.detach().to("cpu", torch.float32).contiguous().numpy()
            student.write(w)
            student.zero_grad()
            xd = x.detach().to(torch.float32).contiguous()
            td = target.detach().to(torch.float32).contiguous()
            loss = student.loss_grad(xd.data_ptr(), td.data_ptr(), int(x.shape[0]), float(sigma))
            g = torch.from_numpy(student.grads().astype(np.float32)).to(weights.device)
            student.zero_grad()
            ctx.save_for_backward(g)
            return torch.tensor(loss, dtype=weights.dtype, device=weights.device)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g.to(grad_out.dtype), None, None, None, None

    return StudentLoss


_CACHE = {}


def student_loss(weights, x, target, sigma: float, student):
    """Loss of the library student as a differentiable function of weights."""
    if "fn" not in _CACHE:
        _CACHE["fn"] = _make()
    return _CACHE["fn"].apply(weights, x, target, sigma, student)
