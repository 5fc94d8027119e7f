"""Additive model (Prop. 5.1, Sec. 5) on the path that builds the 2-D pair blocks from one
partition per first coordinate (owners of two grid rows, exact bucket sizes), against
the oracle.

Cases: tile loads by bulk copy (n a multiple of 4) and by plain loads (other n); the
256-node grid of m = 64 and a 64-node grid (m = 10, owners of two 64-node rows);
d from 2 (one pair, no next-coordinate count) to 10 (nine partners in one partition);
points crowded into a few grid rows of the first coordinates, so that the owners'
buckets are far from equal (the exact counts must still place every point).
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


def unique_part(theta, d, m):
    """Coefficients with k != 0 and the sum of the intercepts (the intercept columns of
    the block Gram coincide, so their differences are fixed only by lambda)."""
    th = np.asarray(theta).reshape(d, 2 * m + 1)
    return np.concatenate([np.delete(th, m, axis=1).ravel(), [th[:, m].sum()]])


def check(X, y, m, lam, eps=1e-6, tol=1e-5):
    d = X.shape[0]
    th = fk.fk_fit_additive(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), m, [lam], eps,
                            "mixed").cpu().numpy()[0, 0]
    Xo, yo = X.astype(np.float64), y.astype(np.float64)
    tho = O.fit_additive(Xo, yo, m, lam)
    assert rel(unique_part(th, d, m), unique_part(tho, d, m)) <= tol
    Xq = S.uniform_points(2000, d, 77).astype(np.float32)
    f = fk.fk_predict(torch.from_numpy(th).cuda(), torch.from_numpy(Xq).cuda(), m, eps, "mixed",
                      additive=True).cpu().numpy()[0]
    assert rel(f, O.predict_additive(tho, Xq.astype(np.float64), m)) <= tol


@pytest.mark.parametrize("d,m,n", [(8, 64, 40000),    # bulk-copy tiles, 256-node grid
                                   (8, 64, 40003),    # plain loads
                                   (5, 10, 24000),    # 64-node grid
                                   (2, 20, 12000),    # one pair
                                   (10, 8, 16000)])   # nine partners of coordinate 0
def test_additive_rowpairs_match_oracle(d, m, n):
    X, y = S.wl4_additive(n, d=d, dtype=np.float32)
    check(X, y, m, 1e-3)


def test_additive_rowpairs_crowded_rows():
    d, m, n = 4, 16, 32000
    X, y = S.wl4_additive(n, d=d, dtype=np.float32)
    g = np.random.default_rng(5)
    # three quarters of the points in a band of a few grid rows of coordinates 0 and 1
    crowd = g.random(n) < 0.75
    X[0, crowd] = (0.3 + 0.02 * g.random(crowd.sum())).astype(np.float32)
    X[1, crowd] = (-1.0 + 0.02 * g.random(crowd.sum())).astype(np.float32)
    y = np.ascontiguousarray(y.astype(np.float32))
    # lambda = 0.1: the crowded rows make the block Gram ill-conditioned, which would
    # amplify the NUFFT tolerance beyond the gate at small lambda (this case is about
    # every point reaching its bucket)
    check(np.ascontiguousarray(X), y, m, 1e-1)
