"""Additive model (Prop. 5.1) on the GPU against the oracle's block Gram and
brute-force additive kernel ridge regression."""
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
    """What the additive estimator determines well: every coefficient with k != 0 and
    the sum of the d intercepts.  The intercept columns of Sigma coincide, so the
    differences between intercepts are only fixed by lambda (condition ~ d / lambda)."""
    th = np.asarray(theta).reshape(d, 2 * m + 1)
    return np.concatenate([np.delete(th, m, axis=1).ravel(), [th[:, m].sum()]])


@pytest.mark.parametrize("precision,eps,tol,d,m,n", [("fp64", 1e-13, 1e-10, 3, 6, 5003),  # cond ~ d / lambda
                                                      ("mixed", 1e-6, 1e-5, 8, 20, 20011),
                                                      ("mixed", 1e-6, 1e-5, 8, 64, 30011)])
def test_fit_additive_matches_oracle(precision, eps, tol, d, m, n):
    nd = np.float64 if precision == "fp64" else np.float32
    td = torch.float64 if precision == "fp64" else torch.float32
    X, y = S.wl4_additive(n, d=d, dtype=nd)
    lams = [1e-3, 2.3e-7 * 1e3]
    th = fk.fk_fit_additive(torch.from_numpy(X).to("cuda", td), torch.from_numpy(y).to("cuda", td), m, lams, eps,
                            precision).cpu().numpy()
    for li, lam in enumerate(lams):
        tho = O.fit_additive(X.astype(np.float64), y.astype(np.float64), m, lam)
        assert rel(unique_part(th[li, 0], d, m), unique_part(tho, d, m)) <= tol
        # The intercepts are equal in exact arithmetic: the intercept columns of Sigma
        # coincide, so v = e_(l,0) - e_(l',0) has Sigma v = 0 and (Sigma + lambda I)
        # v = lambda v.  An error E in the computed Sigma (and b) moves theta along v by at
        # most (|E| |theta| + |db|) / lambda, with |E| <= eps |Sigma| and |Sigma| ~ d (the
        # all-intercepts direction); 10x margin.
        ic = th[li, 0].reshape(d, 2 * m + 1)[:, m]
        spread = float(np.max(np.abs(ic - ic.mean())))
        bound = 10 * eps * d * np.linalg.norm(th[li, 0]) / lam
        assert spread <= bound
    Xq = S.uniform_points(3000, d, 42).astype(nd)
    f = fk.fk_predict(torch.from_numpy(th[0]).cuda(), torch.from_numpy(Xq).to("cuda", td), m, eps, precision,
                      additive=True).cpu().numpy()[0]
    fo = O.predict_additive(O.fit_additive(X.astype(np.float64), y.astype(np.float64), m, lams[0]),
                            Xq.astype(np.float64), m)
    assert rel(f, fo) <= tol


def test_additive_matches_bruteforce_krr():
    d, m, lam, n = 3, 4, 1e-3, 800
    X, y = S.wl4_additive(n, d=d, dtype=np.float64)
    th = fk.fk_fit_additive(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), m, [lam], 1e-12, "fp64")
    Xq = S.uniform_points(64, d, 43)
    f = fk.fk_predict(th[0], torch.from_numpy(Xq).cuda(), m, 1e-12, "fp64", additive=True).cpu().numpy()[0]
    assert rel(f, O.additive_krr(X, y, m, lam, Xq)) <= 1e-10
    # intercepts of the d components are equal (the k = 0 columns coincide)
    ic = th[0, 0, :, m].cpu().numpy()
    assert np.max(np.abs(ic - ic[0])) < 1e-10


def test_additive_rejects_zero_lambda():
    X = torch.zeros((2, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(fk.FkError):
        fk.fk_fit_additive(X, X[0], 3, [0.0], 1e-6, "fp64")


def test_additive_fits_from_two_host_threads():
    # the fit forks its pair and 1-D transforms onto side streams of the calling host
    # thread (joined before it returns); two threads fitting at once on their own
    # streams must each get the answer of a fit made alone
    import threading

    d, m, n = 8, 20, 40_000
    X, y = S.wl4_additive(n, d=d, dtype=np.float32)
    lam = 1e-3
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    want = fk.fk_fit_additive(Xd, yd, m, [lam], 1e-6, "mixed").cpu().numpy()[0, 0]
    tho = O.fit_additive(X.astype(np.float64), y.astype(np.float64), m, lam)
    assert rel(unique_part(want, d, m), unique_part(tho, d, m)) <= 1e-5
    out, errs = {}, []

    def worker(k):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                res = [fk.fk_fit_additive(Xd, yd, m, [lam], 1e-6, "mixed") for _ in range(3)]
            s.synchronize()
            out[k] = [r.cpu().numpy()[0, 0] for r in res]
        except Exception as e:  # reported below
            errs.append(e)

    ts = [threading.Thread(target=worker, args=(k,)) for k in range(2)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errs, errs
    for k in range(2):
        for th in out[k]:
            # the 2-D register sums depend on the order in which records reach a cell,
            # so fits agree to the spreading's rounding, not bit for bit
            assert rel(unique_part(th, d, m), unique_part(want, d, m)) <= 1e-6
