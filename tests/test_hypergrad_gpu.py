"""Held-out-loss hypergradients on the GPU against the oracle's adjoint formulas
and against central finite differences of the GPU forward pass.

Workload shape: 2-D physics-informed (t, x) heat prior P = d_t - 0.1 d_xx at reduced
n (the oracle's dense solve and direct sums must finish in seconds)."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

fk = pytest.importorskip("paper_2509_02649_b300")

ALPHA = [[1, 0], [0, 2]]


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def setup(precision, n=6001, nv=2003, m=12):
    nd = np.float64 if precision == "fp64" else np.float32
    td = torch.float64 if precision == "fp64" else torch.float32
    x, y = S.wl3_pik_heat(n, dtype=nd)
    xv, yv = S.wl3_pik_heat(nv, dtype=nd, validation=True)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", td)
    return x, y, xv, yv, dev(x), dev(y), dev(xv), dev(yv), m


@pytest.mark.parametrize("precision,eps,tol", [("fp64", 1e-12, 1e-9), ("mixed", 1e-6, 1e-4)])
def test_hypergrad_matches_oracle_adjoint(precision, eps, tol):
    lam, s, mu, a = 1e-3, 1.0, 1e-2, [1.0, -0.1]
    x, y, xv, yv, xd, yd, xvd, yvd, m = setup(precision)
    W = fk.fk_penalty_weights(2, m, [lam], s=s, mu=mu, alpha=ALPHA, a=a)
    T, b = fk.fk_build_system(xd, yd, m, eps, precision)
    theta = fk.fk_solve(T, W, b, 2, m)[0, 0]
    loss, dW, dY = fk.fk_hypergrad(xd, xvd, yvd, m, T, W[0], theta, eps, precision)
    Wo = O.penalty_pik(2, m, lam, s, mu, ALPHA, a)
    Lo, tho, dWo, dYo = O.hypergradient(x.astype(np.float64), y.astype(np.float64), xv.astype(np.float64),
                                        yv.astype(np.float64), m, Wo)
    assert abs(loss - Lo) <= tol * Lo
    assert rel(dW.cpu().numpy(), dWo) <= tol
    assert rel(dY.cpu().numpy(), dYo) <= tol
    g = fk.fk_penalty_grads(2, m, dW, lam, s=s, mu=mu, alpha=ALPHA, a=a)
    go = O.penalty_param_grads(2, m, lam, s, mu, ALPHA, a, dWo)
    assert abs(g[0] - go["lambda"]) <= tol * abs(go["lambda"])
    assert abs(g[1] - go["s"]) <= tol * abs(go["s"])
    assert abs(g[2] - go["mu"]) <= tol * abs(go["mu"])
    assert np.max(np.abs(np.array(g[3:]) - go["a"]) / np.abs(go["a"])) <= tol


def test_autograd_matches_finite_differences_fp64():
    eps = 1e-12
    x, y, xv, yv, xd, yd, xvd, yvd, m = setup("fp64", n=4001, nv=1501, m=10)
    params = dict(lam=2e-3, s=1.0, mu=3e-2, c=0.1)

    def loss_of(lam, s, mu, c, yy=yd, grad=False):
        lt = torch.tensor(lam, dtype=torch.float64, requires_grad=grad)
        st = torch.tensor(s, dtype=torch.float64, requires_grad=grad)
        mt = torch.tensor(mu, dtype=torch.float64, requires_grad=grad)
        at = torch.tensor([1.0, -c], dtype=torch.float64, requires_grad=grad)
        yq = yy.clone().requires_grad_(grad)
        L = fk.heldout_loss(yq, lt, st, mt, at, xd, xvd, yvd, m, ALPHA, eps, "fp64")
        if grad:
            L.backward()
            return float(L.detach()), lt.grad.item(), st.grad.item(), mt.grad.item(), -at.grad[1].item(), yq.grad
        return float(L)

    L, gl, gs, gm, gc, gy = loss_of(**params, grad=True)

    def fd(name, rel_step=1e-5):
        v = params[name]
        h = rel_step * abs(v)
        up = dict(params, **{name: v + h})
        dn = dict(params, **{name: v - h})
        return (loss_of(**up) - loss_of(**dn)) / (2 * h)

    assert abs(fd("lam") - gl) <= 1e-6 * abs(gl)
    assert abs(fd("s") - gs) <= 1e-6 * abs(gs)
    assert abs(fd("mu") - gm) <= 1e-6 * abs(gm)
    assert abs(fd("c") - gc) <= 1e-6 * abs(gc)   # diffusion coefficient of the heat prior
    gy = gy.cpu().numpy().ravel()
    for i in [3, 777, 2500]:
        h = 1e-3
        yp = yd.clone()
        yp[i] += h
        ym = yd.clone()
        ym[i] -= h
        fdy = (loss_of(**params, yy=yp) - loss_of(**params, yy=ym)) / (2 * h)
        assert abs(fdy - gy[i]) <= 1e-6 * abs(gy[i]) + 1e-14


def test_autograd_forward_only_fits_backward_does_the_adjoint():
    """The forward pass is the fit and the held-out loss; the adjoint solve and the
    type-1 / type-2 pair run in backward (their kernel launches come after forward)."""
    eps = 1e-12
    x, y, xv, yv, xd, yd, xvd, yvd, m = setup("fp64", n=4001, nv=1501, m=10)
    lt = torch.tensor(2e-3, dtype=torch.float64, requires_grad=True)
    st = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    mt = torch.tensor(3e-2, dtype=torch.float64, requires_grad=True)
    at = torch.tensor([1.0, -0.1], dtype=torch.float64, requires_grad=True)
    yq = yd.clone().requires_grad_(True)
    c0 = fk.fk_launch_count()
    L = fk.heldout_loss(yq, lt, st, mt, at, xd, xvd, yvd, m, ALPHA, eps, "fp64")
    c1 = fk.fk_launch_count()
    L.backward()
    c2 = fk.fk_launch_count()
    assert c1 > c0 and c2 - c1 >= 4  # backward: type-1 of r, mode extraction, solve, dW, type-2 at X
    # the forward's loss and the backward's gradients agree with the single-call adjoint
    W = fk.fk_penalty_weights(2, m, [2e-3], s=1.0, mu=3e-2, alpha=ALPHA, a=[1.0, -0.1])
    T, b = fk.fk_build_system(xd, yd, m, eps, "fp64")
    theta = fk.fk_solve(T, W, b, 2, m)[0, 0]
    loss, dW, dY = fk.fk_hypergrad(xd, xvd, yvd, m, T, W[0], theta, eps, "fp64")
    g = fk.fk_penalty_grads(2, m, dW, 2e-3, s=1.0, mu=3e-2, alpha=ALPHA, a=[1.0, -0.1])
    assert abs(float(L.detach()) - loss) <= 1e-12 * loss
    assert abs(lt.grad.item() - g[0]) <= 1e-10 * abs(g[0])
    assert abs(mt.grad.item() - g[2]) <= 1e-10 * abs(g[2])
    assert rel(yq.grad.cpu().numpy(), dY.cpu().numpy()) <= 1e-10


@pytest.mark.parametrize("precision,eps,tol", [("fp64", 1e-12, 1e-10), ("mixed", 1e-6, 1e-5)])
def test_chunked_loss_regenerates_points_and_matches_whole(precision, eps, tol):
    """Training points drawn per chunk from a seed (never held at once) give the same loss
    and hyperparameter gradients as the whole-array form on the same points."""
    td = torch.float64 if precision == "fp64" else torch.float32
    n_chunks, c, m = 4, 3001, 10
    _, _, xv, yv, _, _, xvd, yvd, _ = setup(precision, n=16, nv=1501, m=m)

    def source(i):  # chunk i of the heat workload, drawn on the device from its own seed
        g = torch.Generator(device="cuda")
        g.manual_seed(1000 + i)
        xi = (torch.rand((2, c), generator=g, device="cuda", dtype=torch.float64) * 6.283185307179586
              - 3.141592653589793).to(td)
        yi = (torch.exp(-0.1 * xi[0].double()) * torch.sin(xi[1].double())
              + 0.1 * torch.randn(c, generator=g, device="cuda", dtype=torch.float64)).to(td)
        return xi, yi

    def leaves():
        return [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (2e-3, 1.0, 3e-2)] + \
               [torch.tensor([1.0, -0.1], dtype=torch.float64, requires_grad=True)]

    lt, st, mt, at = leaves()
    Lc = fk.heldout_loss_chunked(source, n_chunks, lt, st, mt, at, xvd, yvd, m, ALPHA, eps, precision)
    Lc.backward()
    parts = [source(i) for i in range(n_chunks)]
    X = torch.cat([p[0] for p in parts], dim=1).contiguous()
    Y = torch.cat([p[1] for p in parts]).contiguous()
    lw, sw, mw, aw = leaves()
    Lw = fk.heldout_loss(Y, lw, sw, mw, aw, X, xvd, yvd, m, ALPHA, eps, precision)
    Lw.backward()
    assert abs(float(Lc.detach()) - float(Lw.detach())) <= tol * float(Lw.detach())
    for a, b in ((lt, lw), (st, sw), (mt, mw)):
        assert abs(a.grad.item() - b.grad.item()) <= tol * abs(b.grad.item())
    assert float((at.grad - aw.grad).abs().max()) <= tol * float(aw.grad.abs().max())
