"""Three-dimensional transforms and fits (the paper's NUFFTs go up to d = 3): type-1,
type-2 and the Sobolev fit against the oracle, on both solver routes."""
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


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


PREC = {"fp64": (torch.float64, np.float64, 1e-12), "mixed": (torch.float32, np.float32, 1e-6)}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kmax,n", [(6, 2000), (3, 333)])
def test_type1_type2_3d(precision, kmax, n):
    td, nd, eps = PREC[precision]
    x = S.uniform_points(n, 3, 51).astype(nd)
    g = np.random.default_rng(2)
    c = g.standard_normal((2, n)).astype(nd)
    out = fk.fk_type1(dev(x, td), dev(c, td), kmax, eps, precision).cpu().numpy()
    want = O.type1(x.astype(np.float64), c.astype(np.float64), kmax)
    for ch in range(2):
        assert rel(out[ch], want[ch]) < 10 * eps
    K = 2 * kmax + 1
    coef = g.standard_normal((1, K ** 3)) + 1j * g.standard_normal((1, K ** 3))
    f = fk.fk_type2(dev(coef, torch.complex128), dev(x, td), kmax, eps, precision).cpu().numpy()
    fw = O.type2(coef[0], x.astype(np.float64), kmax).real
    assert rel(f.ravel(), fw) < 10 * eps


@pytest.mark.parametrize("solver", ["chol", "cg"])
def test_sobolev_fit_3d(solver):
    m, n = 4, 20000
    x = S.uniform_points(n, 3, 52)
    y = np.sin(x[0]) * np.cos(2 * x[1]) + 0.3 * np.sin(x[2]) + 0.05 * np.random.default_rng(3).standard_normal(n)
    opts = fk.default_opts(solver=fk.FK_SOLVER_CHOL if solver == "chol" else fk.FK_SOLVER_CG, cg_tol=1e-13)
    th = fk.fk_fit_sobolev(dev(x, torch.float64), dev(y, torch.float64), m, 1.0, [1e-4, 1e-2], 1e-12, "fp64",
                           opts=opts).cpu().numpy()
    for li, lam in enumerate([1e-4, 1e-2]):
        want = O.fit(x, y, m, O.penalty_sobolev(3, m, lam, 1.0))
        assert rel(th[li, 0], want) < 1e-10
    # predictions (type-2 of the fit) against the oracle's
    xq = S.uniform_points(500, 3, 53)
    f = fk.fk_predict(dev(th[0], torch.complex128), dev(xq, torch.float64), m, 1e-12, "fp64").cpu().numpy().ravel()
    assert rel(f, O.predict(th[0, 0], xq, m)) < 1e-10
