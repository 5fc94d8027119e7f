"""Differentiable held-out loss of the Fourier kernel estimator (autograd form).

HeldOutLoss.apply(y, lam, s, mu, a, x, xv, yv, m, alpha, eps, precision) returns
L = mean((f_hat(xv) - yv)^2) where f_hat is the fit of Eq. 2 on (x, y) with the
penalty W_k = lam (1 + |k|^{2s}) + mu |P(ik)|^2, P(ik) = sum_t a_t prod_l (i k_l)^{alpha_t,l}
(Sec. 3.1, Sec. 4).

* forward: the fit (moments T and right-hand side b by type-1 transforms, the penalty,
  the solve) and the held-out loss (type-2 prediction at xv and the residual), all in
  libfk (fk_build_system, fk_penalty_weights, fk_solve, fk_heldout_loss).  No adjoint
  work happens here, so evaluating the loss alone costs the fit and one prediction.
* backward: the adjoint of Eq. 2 (fk_adjoint: type-1 of the residual, the adjoint solve
  with the fit's matrix, dL/dW), the chain rule to lam, s, mu and each a_t
  (fk_penalty_grads), and, when y needs a gradient, dL/dY by a type-2 transform of the
  adjoint solution at the training points (fk_type2).

heldout_loss_chunked(source, n_chunks, ...) is the same loss with the training points
produced chunk by chunk by `source(i) -> (x_i, y_i)` (for example drawn on the device
from a seed): they are spread onto an accumulator's grids as they come and never held
all at once.  Its backward gives the gradients of lam, s, mu and a; it needs no training
point at all (the adjoint uses the fit's moments T only).

Gradients flow to y (a CUDA tensor), lam, s, mu and each coefficient a_t (0-dim /
1-d tensors; their values are read on the host).
"""
from __future__ import annotations

import torch

from . import _lib as L


def _penalty_args(lam, s, mu, a, alpha):
    lam_v, s_v, mu_v = float(lam), float(s), float(mu)
    a_v = [float(v) for v in a.reshape(-1).tolist()] if a is not None else []
    al = [list(r) for r in alpha] if a_v else []
    return lam_v, s_v, mu_v, a_v, al


def _grads(ctx, go, g):
    gl = torch.tensor(go * g[0], dtype=torch.float64)
    gs = torch.tensor(go * g[1], dtype=torch.float64)
    gm = torch.tensor(go * g[2], dtype=torch.float64)
    ga = None
    if ctx.a_shape is not None:
        ga = torch.tensor([go * v for v in g[3:]], dtype=torch.float64).reshape(ctx.a_shape)
    return gl, gs, gm, ga


class HeldOutLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, lam, s, mu, a, x, xv, yv, m, alpha, eps, precision="mixed"):
        d = x.shape[0] if x.dim() == 2 else 1
        lam_v, s_v, mu_v, a_v, al = _penalty_args(lam, s, mu, a, alpha)
        W = L.fk_penalty_weights(d, m, [lam_v], s=s_v, mu=mu_v, alpha=al, a=a_v, device=y.device)
        T, b = L.fk_build_system(x, y, m, eps, precision)
        theta = L.fk_solve(T, W, b, d, m)[0, 0]
        loss, r = L.fk_heldout_loss(theta, xv, m=m, yv=yv, eps=eps, precision=precision)
        ctx.save_for_backward(T, W[0], theta, r, x, xv)
        ctx.cfg = (d, m, lam_v, s_v, mu_v, a_v, al, eps, precision)
        ctx.n = x.shape[-1]
        ctx.a_shape = None if a is None else a.shape
        ctx.y_dtype, ctx.y_shape = y.dtype, y.shape
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, go):
        T, W, theta, r, x, xv = ctx.saved_tensors
        d, m, lam_v, s_v, mu_v, a_v, al, eps, precision = ctx.cfg
        go = float(go)
        want_y = bool(ctx.needs_input_grad[0])
        # z scaled by 2 go / n: its type-2 sums at the training points are go dL/dY
        dW, zy = L.fk_adjoint(xv, r, T, W, theta, m, eps, precision, zscale=2.0 * go / ctx.n, want_zy=want_y)
        g = L.fk_penalty_grads(d, m, dW, lam_v, s=s_v, mu=mu_v, alpha=al, a=a_v)
        gy = None
        if want_y:
            gy = L.fk_type2(zy, x, m, eps, precision)[0].to(ctx.y_dtype).reshape(ctx.y_shape)
        return (gy,) + _grads(ctx, go, g) + (None,) * 7


class ChunkedHeldOutLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lam, s, mu, a, source, n_chunks, xv, yv, m, alpha, eps, precision="mixed"):
        d = xv.shape[0] if xv.dim() == 2 else 1
        lam_v, s_v, mu_v, a_v, al = _penalty_args(lam, s, mu, a, alpha)
        acc = L.Accumulator(d, m, 1, eps, precision, device=xv.device)
        try:
            for i in range(n_chunks):
                xi, yi = source(i)
                acc.add(xi, yi, keep=False)  # the chunk is not kept: points are never all held
                del xi, yi
            T, b, n = acc.system()
        finally:
            acc.close()
        W = L.fk_penalty_weights(d, m, [lam_v], s=s_v, mu=mu_v, alpha=al, a=a_v, device=xv.device)
        theta = L.fk_solve(T, W, b, d, m)[0, 0]
        loss, r = L.fk_heldout_loss(theta, xv, m=m, yv=yv, eps=eps, precision=precision)
        ctx.save_for_backward(T, W[0], theta, r, xv)
        ctx.cfg = (d, m, lam_v, s_v, mu_v, a_v, al, eps, precision)
        ctx.a_shape = None if a is None else a.shape
        ctx.n = n
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, go):
        T, W, theta, r, xv = ctx.saved_tensors
        d, m, lam_v, s_v, mu_v, a_v, al, eps, precision = ctx.cfg
        go = float(go)
        dW, _ = L.fk_adjoint(xv, r, T, W, theta, m, eps, precision)
        g = L.fk_penalty_grads(d, m, dW, lam_v, s=s_v, mu=mu_v, alpha=al, a=a_v)
        return _grads(ctx, go, g) + (None,) * 8


def heldout_loss(y, lam, s, mu, a, x, xv, yv, m, alpha, eps, precision="mixed"):
    return HeldOutLoss.apply(y, lam, s, mu, a, x, xv, yv, m, alpha, eps, precision)


def heldout_loss_chunked(source, n_chunks, lam, s, mu, a, xv, yv, m, alpha, eps, precision="mixed"):
    return ChunkedHeldOutLoss.apply(lam, s, mu, a, source, n_chunks, xv, yv, m, alpha, eps, precision)
