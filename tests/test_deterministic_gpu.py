"""Deterministic sums (fk_opts.deterministic = 1): T and b must come out bit for bit the
same on repeated runs, for d = 1, 2, 3 and both precisions, and agree with the oracle
within the NUFFT tolerance.  The 64-bit fixed-point sums round each contribution to a
multiple of 2^(e - 61) with n max|strength| <= 2^e, far below eps.
"""
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


@pytest.mark.parametrize("d,m,n,precision,eps", [(2, 12, 40000, "mixed", 1e-6), (2, 8, 20000, "fp64", 1e-12),
                                                 (3, 4, 6000, "fp64", 1e-10), (3, 4, 6000, "mixed", 1e-6),
                                                 (1, 40, 30000, "fp64", 1e-12)])
def test_deterministic_sums_repeat_bitwise_and_match_oracle(d, m, n, precision, eps):
    dt = torch.float64 if precision == "fp64" else torch.float32
    x = torch.from_numpy(S.uniform_points(n, d, 61)).to("cuda", dt)
    y = torch.from_numpy(np.stack([S.noise(n, 1.0, 61, 1), S.noise(n, 0.3, 61, 2)])).to("cuda", dt)
    opts = fk.default_opts(deterministic=1)
    T1, b1 = fk.fk_build_system(x, y, m, eps, precision, opts=opts)
    T2, b2 = fk.fk_build_system(x, y, m, eps, precision, opts=opts)
    assert torch.equal(T1, T2) and torch.equal(b1, b2)
    xo, yo = x.double().cpu().numpy(), y.double().cpu().numpy()
    tol = 10 * eps
    assert rel(T1.cpu().numpy(), O.moments(xo, m)) <= tol
    assert rel(b1.cpu().numpy(), O.rhs(xo, yo, m)) <= tol


def test_deterministic_additive_matches_oracle_and_repeats():
    d, m, n, lam = 4, 10, 12000, 1e-3
    X, y = S.wl4_additive(n, d=d, dtype=np.float32)
    xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    opts = fk.default_opts(deterministic=1)
    th1 = fk.fk_fit_additive(xd, yd, m, [lam], 1e-6, "mixed", opts=opts)
    th2 = fk.fk_fit_additive(xd, yd, m, [lam], 1e-6, "mixed", opts=opts)
    # the block sums repeat bit for bit; the dense solve on them repeats to rounding
    assert float((th1 - th2).abs().max() / th1.abs().max()) <= 1e-13
    tho = O.fit_additive(X.astype(np.float64), y.astype(np.float64), m, lam).reshape(d, 2 * m + 1)
    th = th1[0, 0].cpu().numpy()
    # coefficients with k != 0 and the intercept sum (the intercept differences are set by lambda)
    keep = lambda t: np.concatenate([np.delete(t, m, axis=1).ravel(), [t[:, m].sum()]])
    assert rel(keep(th), keep(tho)) <= 1e-5
