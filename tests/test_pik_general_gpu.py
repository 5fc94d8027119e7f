"""Physics-informed fits on a sub-domain (closed-form box moments) and with
collocation points (§4): the penalty mu D^* C D with a non-diagonal Toeplitz C,
against the oracle's dense solve, on the Cholesky route and on both CG forms."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

fk = pytest.importorskip("paper_2509_02649_b300")

ALPHA2, A2 = [[1, 0], [0, 2]], [1.0, -0.1]


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("d,lo,hi", [(1, -0.4, 1.3), (2, (-1.0, 0.2), (0.7, 2.9)), (2, -math.pi, math.pi)])
def test_box_moments(d, lo, hi):
    m = 9
    c = fk.fk_box_moments(d, m, lo, hi).cpu().numpy()
    want = O.box_moments(d, m, lo, hi)
    assert np.max(np.abs(c - want)) < 1e-14


@pytest.mark.parametrize("solver", ["chol", "cg"])
@pytest.mark.parametrize("precision,eps,tol", [("fp64", 1e-12, 1e-9), ("mixed", 1e-6, 1e-5)])
def test_subdomain_fit_2d(solver, precision, eps, tol):
    m, n = 8, 20000
    lo, hi = (-1.2, -0.3), (0.9, 1.4)
    x, y = S.wl3_pik_heat(n, dtype=np.float64)
    td = torch.float64 if precision == "fp64" else torch.float32
    xn = x.astype(np.float64) if precision == "fp64" else x.astype(np.float32).astype(np.float64)
    yn = y.astype(np.float64) if precision == "fp64" else y.astype(np.float32).astype(np.float64)
    c = fk.fk_box_moments(2, m, lo, hi)
    opts = fk.default_opts(solver=fk.FK_SOLVER_CHOL if solver == "chol" else fk.FK_SOLVER_CG, cg_tol=1e-13)
    th = fk.fk_fit_pik_general(dev(xn, td), dev(yn, td), m, 1.0, 1e-4, 0.05, ALPHA2, A2, c, eps, precision,
                               opts=opts)
    Pen = O.penalty_pik_general(2, m, 1e-4, 1.0, 0.05, ALPHA2, A2, O.box_moments(2, m, lo, hi))
    want = O.fit_penalised(xn, yn, m, Pen)
    assert rel(th.cpu().numpy()[0], want) < tol


def test_subdomain_fit_1d_cg():
    # the multi-launch 1-D CG with the operator's second circulant product
    m, n = 40, 30000
    x, y = S.wl1_sobolev_1d(n)
    lo, hi = -0.5, 2.0
    c = fk.fk_box_moments(1, m, lo, hi)
    opts = fk.default_opts(solver=fk.FK_SOLVER_CG, cg_tol=1e-13)
    th, rep = fk.fk_fit_pik_general(dev(x, torch.float64), dev(y, torch.float64), m, 1.0, 1e-5, 0.2, [[1], [0]],
                                    [1.0, -1.0], c, 1e-12, "fp64", opts=opts, report=True)
    Pen = O.penalty_pik_general(1, m, 1e-5, 1.0, 0.2, [[1], [0]], [1.0, -1.0], O.box_moments(1, m, lo, hi))
    want = O.fit_penalised(x, y, m, Pen)
    assert rep["cg_iters"] > 0
    assert rel(th.cpu().numpy()[0], want) < 1e-9


def test_collocation_fit_2d():
    m, n, nr = 6, 15000, 3000
    x, y = S.wl3_pik_heat(n, dtype=np.float64)
    xr = S.uniform_points(nr, 2, 77) * 0.4  # collocation points in a sub-box
    c, _ = fk.fk_build_system(dev(xr, torch.float64), None, 2 * 0 + m, 1e-12, "fp64")
    want_c = O.moments(xr, m)
    assert rel(c.cpu().numpy(), want_c) < 1e-10
    th = fk.fk_fit_pik_general(dev(x, torch.float64), dev(y, torch.float64), m, 1.0, 1e-3, 0.1, ALPHA2, A2, c,
                               1e-12, "fp64")
    Pen = O.penalty_pik_general(2, m, 1e-3, 1.0, 0.1, ALPHA2, A2, want_c)
    want = O.fit_penalised(x, y, m, Pen)
    assert rel(th.cpu().numpy()[0], want) < 1e-9


def test_full_period_reduces_to_diagonal_penalty():
    m, n = 10, 12000
    x, y = S.wl3_pik_heat(n, dtype=np.float64)
    c = fk.fk_box_moments(2, m, -math.pi, math.pi)
    X, Y = dev(x, torch.float64), dev(y, torch.float64)
    for solver in (fk.FK_SOLVER_CHOL, fk.FK_SOLVER_CG):
        opts = fk.default_opts(solver=solver, cg_tol=1e-13)
        g = fk.fk_fit_pik_general(X, Y, m, 1.0, 1e-4, 0.05, ALPHA2, A2, c, 1e-12, "fp64", opts=opts)
        p = fk.fk_fit_pik(X, Y, m, 1.0, 1e-4, 0.05, ALPHA2, A2, 1e-12, "fp64", opts=opts)
        assert rel(g.cpu().numpy(), p.cpu().numpy()) < 1e-10


def test_paper_one_dimensional_example():
    # §4's example: X ~ U(0, 1) (L = pi/2, so the library's coordinates are X itself),
    # Y = exp(X) + N(0, 1), prior f' - f = 0 on Omega = (0, 1), m = n^(1/3), lambda =
    # n^(-2/3), mu = 1; the fit recovers exp on (0, 1)
    n = 1_000_000
    g = torch.Generator(device="cuda")
    g.manual_seed(123)
    x = torch.rand((1, n), generator=g, device="cuda", dtype=torch.float64)
    y = torch.exp(x[0]) + torch.randn(n, generator=g, device="cuda", dtype=torch.float64)
    m = int(round(n ** (1 / 3)))
    c = fk.fk_box_moments(1, m, 0.0, 1.0)
    th = fk.fk_fit_pik_general(x, y, m, 1.0, n ** (-2 / 3), 1.0, [[1], [0]], [1.0, -1.0], c, 1e-9, "fp64")
    xq = torch.linspace(0.01, 0.99, 2000, device="cuda", dtype=torch.float64)[None, :]
    f = fk.fk_predict(th, xq, m, 1e-9, "fp64").reshape(-1).cpu().numpy()
    err = np.sqrt(np.mean((f - np.exp(xq[0].cpu().numpy())) ** 2))
    assert err < 0.02, err
