"""Differentiable held-out loss of the Fourier kernel estimator (autograd form).

HeldOutLoss.apply(y, lam, s, mu, a, x, xv, yv, m, alpha, eps, precision) returns
L = mean((f_hat(xv) - yv)^2) where f_hat is the fit of Eq. 2 on (x, y) with the
penalty W_k = lam (1 + |k|^{2s}) + mu |P(ik)|^2, P(ik) = sum_t a_t prod_l (i k_l)^{alpha_t,l}
(Sec. 3.1, Sec. 4).  Every numerical step runs in libfk: the forward pass builds T and
b, solves, and calls the adjoint kernels (fk_hypergrad, fk_penalty_grads), whose
results the backward pass only scales by the incoming gradient.

Gradients flow to y (a CUDA tensor), lam, s, mu and each coefficient a_t (0-dim /
1-d tensors; their values are read on the host).
"""
from __future__ import annotations

import torch

from . import _lib as L


class HeldOutLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, lam, s, mu, a, x, xv, yv, m, alpha, eps, precision="mixed"):
        d = x.shape[0] if x.dim() == 2 else 1
        lam_v, s_v, mu_v = float(lam), float(s), float(mu)
        a_v = [float(v) for v in a.reshape(-1).tolist()] if a is not None else []
        al = [list(r) for r in alpha] if a_v else []
        W = L.fk_penalty_weights(d, m, [lam_v], s=s_v, mu=mu_v, alpha=al, a=a_v, device=y.device)
        T, b = L.fk_build_system(x, y, m, eps, precision)
        theta = L.fk_solve(T, W, b, d, m)[0, 0]
        # dL/dY (one type-2 pass over the training points and n doubles) only when asked
        loss, dW, dY = L.fk_hypergrad(x, xv, yv, m, T, W[0], theta, eps, precision,
                                      want_dy=bool(ctx.needs_input_grad[0]))
        g = L.fk_penalty_grads(d, m, dW, lam_v, s=s_v, mu=mu_v, alpha=al, a=a_v)
        ctx.save_for_backward(dY)
        ctx.pgrads = g
        ctx.a_shape = None if a is None else a.shape
        ctx.dtypes = (y.dtype,)
        ctx.y_shape = y.shape
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, go):
        (dY,) = ctx.saved_tensors
        g = ctx.pgrads
        go = float(go)
        gy = (go * dY).to(ctx.dtypes[0]).reshape(ctx.y_shape) if (ctx.needs_input_grad[0] and dY is not None) else None
        gl = torch.tensor(go * g[0], dtype=torch.float64)
        gs = torch.tensor(go * g[1], dtype=torch.float64)
        gm = torch.tensor(go * g[2], dtype=torch.float64)
        ga = None
        if ctx.a_shape is not None:
            ga = torch.tensor([go * v for v in g[3:]], dtype=torch.float64).reshape(ctx.a_shape)
        return gy, gl, gs, gm, ga, None, None, None, None, None, None, None


def heldout_loss(y, lam, s, mu, a, x, xv, yv, m, alpha, eps, precision="mixed"):
    return HeldOutLoss.apply(y, lam, s, mu, a, x, xv, yv, m, alpha, eps, precision)
