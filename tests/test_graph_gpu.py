"""Capture of library calls into one CUDA graph: a replay on new data written into the
captured buffers must give what a direct call gives on that data; device-side
conditions surface through the graph's status; calls that need a host round trip
refuse to be recorded and leave the stream usable."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

fk = pytest.importorskip("paper_2509_02649_b300")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def fill_uniform(t, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    t.copy_(torch.rand(t.shape, generator=g, device="cuda", dtype=t.dtype) * (2 * math.pi) - math.pi)


def fill_normal(t, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    t.copy_(torch.randn(t.shape, generator=g, device="cuda", dtype=t.dtype))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_additive_fit_replays_on_new_data(precision):
    n, d, m, lam = 30_000, 4, 12, 1e-4
    dt = torch.float32 if precision == "mixed" else torch.float64
    eps = 1e-6 if precision == "mixed" else 1e-12
    x = torch.empty((d, n), dtype=dt, device="cuda")
    y = torch.empty((1, n), dtype=dt, device="cuda")
    theta = torch.empty((1, 1, d, 2 * m + 1), dtype=torch.complex128, device="cuda")
    fill_uniform(x, 1)
    fill_normal(y, 2)
    torch.cuda.synchronize()
    with fk.capture() as g:
        fk.fk_fit_additive(x, y, m, [lam], eps, precision, out=theta)
    for seed in (3, 5):
        fill_uniform(x, seed)
        fill_normal(y, seed + 1)
        y += torch.sin(x[0:1])
        torch.cuda.synchronize()
        g.launch()
        g.status()
        want = fk.fk_fit_additive(x, y, m, [lam], eps, precision)
        torch.cuda.synchronize()
        # what the estimator determines (the intercepts only through their sum): the
        # mixed path's fp32 cell sums depend on the order points reach a cell, which
        # differs from run to run, so two mixed runs agree to fp32 rounding
        a = theta.reshape(d, 2 * m + 1).cpu().numpy()
        w = want.reshape(d, 2 * m + 1).cpu().numpy()
        nz = np.ones(2 * m + 1, dtype=bool)
        nz[m] = False
        tol = 1e-6 if precision == "mixed" else 1e-11
        assert rel(a[:, nz], w[:, nz]) < tol
        assert abs(a[:, m].sum() - w[:, m].sum()) < tol * np.abs(w).max()
    # and against the oracle on the last data (non-intercept coefficients, their sum)
    th = theta.reshape(d, 2 * m + 1).cpu().numpy()
    tho = O.fit_additive(x.double().cpu().numpy(), y.double().cpu().numpy()[0], m, lam).reshape(d, 2 * m + 1)
    nz = np.ones(2 * m + 1, dtype=bool)
    nz[m] = False
    assert rel(th[:, nz], tho[:, nz]) < (1e-5 if precision == "mixed" else 1e-9)
    g.close()


def test_sobolev_cholesky_fit_and_prediction_replay():
    n, m = 20_000, 10
    x = torch.empty((2, n), dtype=torch.float32, device="cuda")
    y = torch.empty((2, n), dtype=torch.float32, device="cuda")
    xq = torch.empty((2, 5000), dtype=torch.float32, device="cuda")
    theta = torch.empty((3, 2, (2 * m + 1) ** 2), dtype=torch.complex128, device="cuda")
    f = torch.empty((6, 5000), dtype=torch.float64, device="cuda")
    opts = fk.default_opts(solver=fk.FK_SOLVER_CHOL)
    lams = [1e-2, 1e-4, 1e-6]
    fill_uniform(x, 11)
    fill_normal(y, 12)
    fill_uniform(xq, 13)
    torch.cuda.synchronize()
    with fk.capture() as g:
        fk.fk_fit_sobolev(x, y, m, 2.0, lams, 1e-6, "mixed", opts=opts, out=theta)
        fk.fk_predict(theta, xq, m, 1e-6, "mixed", out=f)
    for seed in (21, 31):
        fill_uniform(x, seed)
        fill_normal(y, seed + 1)
        y += torch.exp(-(x ** 2).sum(0))
        fill_uniform(xq, seed + 2)
        torch.cuda.synchronize()
        g.launch()
        g.status()
        th_want = fk.fk_fit_sobolev(x, y, m, 2.0, lams, 1e-6, "mixed", opts=opts)
        f_want = fk.fk_predict(th_want, xq, m, 1e-6, "mixed")
        torch.cuda.synchronize()
        # the mixed path's fp32 cell sums depend on the order points reach a cell
        assert rel(theta.cpu().numpy(), th_want.cpu().numpy()) < 1e-6
        assert rel(f.cpu().numpy(), f_want.cpu().numpy()) < 1e-6
    g.close()


def test_replay_reports_range_error_then_recovers():
    n, m = 4096, 8
    x = torch.empty((1, n), dtype=torch.float32, device="cuda")
    y = torch.ones((1, n), dtype=torch.float32, device="cuda")
    T = torch.empty(4 * m + 1, dtype=torch.complex128, device="cuda")
    b = torch.empty((1, 2 * m + 1), dtype=torch.complex128, device="cuda")
    fill_uniform(x, 41)
    torch.cuda.synchronize()
    with fk.capture() as g:
        fk.fk_build_system(x, y, m, 1e-6, "mixed", out=(T, b))
    g.launch()
    g.status()
    x[0, 100] = 10.0  # outside [-3 pi, 3 pi)
    torch.cuda.synchronize()
    g.launch()
    with pytest.raises(fk.FkError) as e:
        g.status()
    assert e.value.name == "FK_ERANGE"
    fill_uniform(x, 42)
    torch.cuda.synchronize()
    g.launch()
    g.status()  # the flag word is cleared at the start of every replay
    Tw, bw = fk.fk_build_system(x, y, m, 1e-6, "mixed")
    torch.cuda.synchronize()
    # 1-D mixed: integer sums, independent of the order of the additions
    assert torch.equal(T, Tw) and torch.equal(b, bw)
    g.close()


def test_uncapturable_calls_refuse_and_leave_the_stream_usable():
    n, m = 20_000, 600  # 1-D, D = 1201 > 1024: the automatic solver is the batched 1-D CG
    x = torch.empty((1, n), dtype=torch.float32, device="cuda")
    y = torch.empty((1, n), dtype=torch.float32, device="cuda")
    fill_uniform(x, 51)
    fill_normal(y, 52)
    out = torch.empty((1, 1, 2 * m + 1), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(fk.FkError) as e:
        with fk.capture():
            fk.fk_fit_sobolev(x, y, m, 2.0, [1e-4], 1e-6, "mixed", out=out)
    assert e.value.name == "FK_EINVAL"
    with pytest.raises(fk.FkError):
        with fk.capture():
            fk.fk_fit_sobolev(x, y, 5, 2.0, [1e-4], 1e-6, "mixed", out=torch.empty(
                (1, 1, 11), dtype=torch.complex128, device="cuda"), report=True)
    with pytest.raises(ValueError):
        with fk.capture():
            fk.fk_fit_sobolev(x, y, 5, 2.0, [1e-4], 1e-6, "mixed")  # no out=
    # direct calls still work, on any stream
    th = fk.fk_fit_sobolev(x, y, m, 2.0, [1e-4], 1e-6, "mixed")
    torch.cuda.synchronize()
    assert torch.isfinite(th.real).all()


def test_two_d_cg_fit_replays_with_kernel_timing():
    # the 2-D single-launch CG (D = 41^2 > 1024) records into the graph; its convergence
    # failure reaches the graph's status as FK_ENOCONV
    n, m = 400_000, 20
    x = torch.empty((2, n), dtype=torch.float32, device="cuda")
    y = torch.empty((1, n), dtype=torch.float32, device="cuda")
    theta = torch.empty((1, 1, (2 * m + 1) ** 2), dtype=torch.complex128, device="cuda")
    fill_uniform(x, 91)
    fill_normal(y, 92)
    y.mul_(0.05).add_(torch.exp(-(x ** 2).sum(0)))
    torch.cuda.synchronize()
    with fk.capture() as g:
        fk.fk_fit_sobolev(x, y, m, 2.0, [1e-6], 1e-6, "mixed", out=theta)
    g.launch()
    g.status()
    assert g.kernel_ms() > 0.0
    want = fk.fk_fit_sobolev(x, y, m, 2.0, [1e-6], 1e-6, "mixed")
    torch.cuda.synchronize()
    assert rel(theta.cpu().numpy(), want.cpu().numpy()) < 1e-6
    g.close()
    opts = fk.default_opts(cg_maxit=1, cg_tol=1e-15)
    with fk.capture() as g2:
        fk.fk_fit_sobolev(x, y, m, 2.0, [1e-6], 1e-6, "mixed", opts=opts, out=theta)
    g2.launch()
    with pytest.raises(fk.FkError) as e:
        g2.status()
    assert e.value.name == "FK_ENOCONV"
    g2.close()


def test_graph_of_many_small_fits_matches_direct_calls():
    # a batch of independent small fits (e.g. the 1-D FP64 workload at n = 1e5) as one graph
    n, m, k = 100_000, 50, 8
    xs = [torch.empty((1, n), dtype=torch.float64, device="cuda") for _ in range(k)]
    ys = [torch.empty((1, n), dtype=torch.float64, device="cuda") for _ in range(k)]
    outs = [torch.empty((1, 1, 2 * m + 1), dtype=torch.complex128, device="cuda") for _ in range(k)]
    for i in range(k):
        fill_uniform(xs[i], 60 + i)
        fill_normal(ys[i], 80 + i)
        ys[i].mul_(0.1).add_(torch.sin(3 * xs[i]) + 0.5 * torch.cos(7 * xs[i]))
    torch.cuda.synchronize()
    with fk.capture() as g:
        for i in range(k):
            fk.fk_fit_sobolev(xs[i], ys[i], m, 1.0, [1e-4], 1e-12, "fp64", out=outs[i])
    g.launch()
    g.status()
    for i in range(k):
        want = fk.fk_fit_sobolev(xs[i], ys[i], m, 1.0, [1e-4], 1e-12, "fp64")
        torch.cuda.synchronize()
        assert rel(outs[i].cpu().numpy(), want.cpu().numpy()) < 1e-11  # fp64 atomics: order only
    x0 = xs[0].cpu().numpy()
    y0 = ys[0].cpu().numpy()
    tho = O.fit(x0, y0[0], m, O.penalty_sobolev(1, m, 1e-4, 1.0))
    assert rel(outs[0].cpu().numpy()[0, 0], tho) < 1e-10
    g.close()
