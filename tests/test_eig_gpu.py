"""Eigen route for sweeps over lambda (fk_opts.solver = FK_SOLVER_EIG, Sec. 5 grid search):
one Hermitian eigendecomposition (parallel cyclic Jacobi, FP64) serves every penalty
lambda_l S^2 of a sweep.  Each fit of the sweep must match the oracle's dense solve of
the same system, and the Cholesky route, for Sobolev (scaled form), low-bias and
additive penalties."""
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


EIG = dict(solver=3)


@pytest.mark.parametrize("d,m,n,precision,eps,tol,penalty", [
    (1, 50, 20000, "fp64", 1e-12, 1e-10, 0),   # Sobolev, D = 101
    (1, 50, 20000, "fp64", 1e-12, 1e-10, 1),   # low-bias
    (2, 8, 30000, "mixed", 1e-6, 1e-5, 0),     # Sobolev, D = 289
])
def test_eig_sweep_matches_oracle_and_cholesky(d, m, n, precision, eps, tol, penalty):
    nd = np.float64 if precision == "fp64" else np.float32
    td = torch.float64 if precision == "fp64" else torch.float32
    if d == 1:
        x, y = S.wl1_sobolev_1d(n, dtype=nd)
    else:
        x, y = S.wl2_sobolev_2d(n, dtype=nd)
    xd, yd = torch.from_numpy(x).to("cuda", td), torch.from_numpy(y).to("cuda", td)
    s = 1.0 if d == 1 else 2.0
    lams = list(np.logspace(-7, -1, 9))
    th = fk.fk_fit_sobolev(xd, yd, m, s, lams, eps, precision, penalty=penalty,
                           opts=fk.default_opts(**EIG)).cpu().numpy()
    thc = fk.fk_fit_sobolev(xd, yd, m, s, lams, eps, precision, penalty=penalty,
                            opts=fk.default_opts(solver=1)).cpu().numpy()
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    for li, lam in enumerate(lams):
        W = O.penalty_sobolev(d, m, lam, s) if penalty == 0 else O.penalty_lowbias(d, m, lam)
        tho = O.fit(x64, y64, m, W)
        assert rel(th[li, 0], tho) <= tol, (li, lam)
        assert rel(th[li, 0], thc[li, 0]) <= tol


def test_eig_additive_lambda_sweep():
    d, m, n = 3, 6, 8000
    X, y = S.wl4_additive(n, d=d, dtype=np.float64)
    lams = list(np.logspace(-4, -1, 7))
    xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    th = fk.fk_fit_additive(xd, yd, m, lams, 1e-12, "fp64", opts=fk.default_opts(**EIG)).cpu().numpy()
    thc = fk.fk_fit_additive(xd, yd, m, lams, 1e-12, "fp64", opts=fk.default_opts(solver=1)).cpu().numpy()
    keep = lambda t: np.concatenate([np.delete(t.reshape(d, 2 * m + 1), m, axis=1).ravel(),
                                     [t.reshape(d, 2 * m + 1)[:, m].sum()]])
    for li, lam in enumerate(lams):
        tho = O.fit_additive(X, y, m, lam)
        assert rel(keep(th[li, 0]), keep(tho)) <= 1e-9, (li, lam)
        assert rel(keep(th[li, 0]), keep(thc[li, 0])) <= 1e-9


def test_eig_rejects_penalties_not_of_the_sweep_form():
    x, y = S.wl2_sobolev_2d(4000, dtype=np.float32)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    with pytest.raises(fk.FkError) as e:
        fk.fk_fit_pik(xd, yd, 6, 1.0, 1e-3, 1e-2, [[1, 0], [0, 2]], [1.0, -0.1], 1e-6, "mixed",
                      opts=fk.default_opts(**EIG))
    assert e.value.name == "FK_EINVAL"
    with pytest.raises(fk.FkError) as e:
        fk.fk_fit_sobolev(xd, yd, 6, 2.0, [1e-3], 1e-6, "mixed", opts=fk.default_opts(solver=3, sobolev_c0=0.0))
    assert e.value.name == "FK_EINVAL"
