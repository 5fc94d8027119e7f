"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Tolerances (normwise relative l2, per result vector):
  * NUFFT building blocks: <= 10 * eps (eps = requested NUFFT tolerance);
  * fits and predictions: <= 1e-10 on the FP64 path (eps = 1e-12), <= 1e-5 on the
    mixed path (eps = 1e-6).
The oracle always receives exactly the points the GPU sees (fp32 points are
widened to fp64 exactly).
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


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().cpu().numpy()


PREC = {"fp64": (torch.float64, np.float64), "mixed": (torch.float32, np.float32)}


@pytest.mark.parametrize("precision,eps", [("fp64", 1e-12), ("fp64", 1e-9), ("mixed", 1e-6), ("mixed", 1e-4)])
@pytest.mark.parametrize("d,kmax,n", [(1, 100, 3001), (1, 7, 517), (2, 20, 4099), (2, 3, 1000)])
def test_type1_matches_direct_sums(precision, eps, d, kmax, n):
    td, nd = PREC[precision]
    x = S.uniform_points(n, d, 21).astype(nd)
    c = S.noise(n, 1.0, 21, 3).astype(nd)
    got = host(fk.fk_type1(dev(x, td), dev(c, td), kmax, eps, precision))[0]
    want = O.type1(x.astype(np.float64), c.astype(np.float64), kmax)
    assert rel(got, want) <= 10 * eps


@pytest.mark.parametrize("precision,eps", [("fp64", 1e-12), ("mixed", 1e-6)])
@pytest.mark.parametrize("d,kmax,n", [(1, 50, 2001), (2, 12, 3001)])
def test_type2_matches_direct_sums(precision, eps, d, kmax, n):
    td, nd = PREC[precision]
    x = S.uniform_points(n, d, 22).astype(nd)
    g = np.random.default_rng(5)
    D = (2 * kmax + 1) ** d
    coef = g.standard_normal((2, D)) + 1j * g.standard_normal((2, D))
    got = host(fk.fk_type2(torch.from_numpy(coef).cuda(), dev(x, td), kmax, eps, precision))
    for s_ in range(2):
        want = O.type2(coef[s_], x.astype(np.float64), kmax)
        assert rel(got[s_], want.real) <= 10 * eps * np.linalg.norm(want) / np.linalg.norm(want.real)


def test_type1_type2_adjoint_on_gpu():
    n, kmax = 2000, 9
    x = S.uniform_points(n, 2, 23)
    g = np.random.default_rng(6)
    c = g.standard_normal(n)
    th = g.standard_normal((2 * kmax + 1) ** 2) + 1j * g.standard_normal((2 * kmax + 1) ** 2)
    F = host(fk.fk_type1(dev(x, torch.float64), dev(c, torch.float64), kmax, 1e-12, "fp64"))[0]
    f = host(fk.fk_type2(torch.from_numpy(th).cuda(), dev(x, torch.float64), kmax, 1e-12, "fp64"))[0]
    # <type1(c), th> = <c, type2(th)>: the real parts agree (c real)
    assert abs(np.vdot(F, th).real - np.dot(c, f)) < 1e-10 * abs(np.dot(c, f))


@pytest.mark.parametrize("precision,eps,tol", [("fp64", 1e-12, 1e-10), ("mixed", 1e-6, 1e-5)])
def test_build_system_moments_and_rhs(precision, eps, tol):
    td, nd = PREC[precision]
    x, y = S.wl2_sobolev_2d(20011, dtype=nd)
    m = 12
    T, b = fk.fk_build_system(dev(x, td), dev(y, td), m, eps, precision)
    To = O.moments(x.astype(np.float64), m)
    bo = O.rhs(x.astype(np.float64), y.astype(np.float64), m)
    assert rel(host(T), To) <= tol
    assert rel(host(b)[0], bo) <= tol
    # invariants on the GPU result: T_0 = 1, Hermitian symmetry
    Tg = host(T).reshape(4 * m + 1, 4 * m + 1)
    assert abs(Tg[2 * m, 2 * m] - 1.0) < 10 * eps
    assert np.max(np.abs(Tg[::-1, ::-1] - np.conj(Tg))) < 10 * eps


def test_fit_sobolev_1d_fp64_config1():
    # 1-D Sobolev regression, plain FP64: n = 1e5, m = 50, s = 1, lambda = 1e-4, eps = 1e-12
    m, s, lam, eps = 50, 1.0, 1e-4, 1e-12
    x, y = S.wl1_sobolev_1d(100000)
    th = host(fk.fk_fit_sobolev(dev(x, torch.float64), dev(y, torch.float64), m, s, [lam], eps, "fp64"))[0, 0]
    W = O.penalty_sobolev(1, m, lam, s)
    tho = O.fit(x, y, m, W)
    assert rel(th, tho) <= 1e-10
    xq = S.uniform_points(10000, 1, 24)
    f = host(fk.fk_predict(torch.from_numpy(th).cuda(), dev(xq, torch.float64), m, eps, "fp64"))[0]
    assert rel(f, O.predict(tho, xq, m)) <= 1e-10


def test_fit_matches_bruteforce_krr_n2000():
    m, s, lam, eps = 50, 1.0, 1e-4, 1e-12
    x, y = S.wl1_sobolev_1d(2000)
    W = O.penalty_sobolev(1, m, lam, s)
    xq = S.uniform_points(64, 1, 25)
    fq, th_krr = O.krr_bruteforce(x, y, m, W, xq)
    th = host(fk.fk_fit_sobolev(dev(x, torch.float64), dev(y, torch.float64), m, s, [lam], eps, "fp64"))[0, 0]
    assert rel(th, th_krr) <= 1e-10
    f = host(fk.fk_predict(torch.from_numpy(th).cuda(), dev(xq, torch.float64), m, eps, "fp64"))[0]
    assert rel(f, fq) <= 1e-10


@pytest.mark.parametrize("precision,eps,tol", [("mixed", 1e-6, 1e-5), ("fp64", 1e-12, 1e-10)])
def test_fit_sobolev_2d_config2_shape(precision, eps, tol):
    # 2-D Sobolev at reduced n: m = 32 (65 x 65 modes, 129 x 129 moments), s = 2, lambda = 1e-6
    td, nd = PREC[precision]
    m, s, lam = 32, 2.0, 1e-6
    x, y = S.wl2_sobolev_2d(30011, dtype=nd)
    th, rep = fk.fk_fit_sobolev(dev(x, td), dev(y, td), m, s, [lam], eps, precision, report=True)
    th = host(th)[0, 0]
    tho = O.fit(x.astype(np.float64), y.astype(np.float64), m, O.penalty_sobolev(2, m, lam, s))
    assert rel(th, tho) <= tol
    xq = S.uniform_points(5000, 2, 26).astype(nd)
    f = host(fk.fk_predict(torch.from_numpy(th).cuda(), dev(xq, td), m, eps, precision))[0]
    assert rel(f, O.predict(tho, xq.astype(np.float64), m)) <= tol
    assert rep["rel_residual"] < 1e-11


def test_fit_pik_heat_config3_shape():
    m, s, lam, mu, eps = 25, 1.0, 1e-8, 1e-2, 1e-6
    alpha, a = [[1, 0], [0, 2]], [1.0, -0.1]
    x, y = S.wl3_pik_heat(20011, dtype=np.float32)
    th = host(fk.fk_fit_pik(dev(x, torch.float32), dev(y, torch.float32), m, s, lam, mu, alpha, a, eps, "mixed"))[0]
    W = O.penalty_pik(2, m, lam, s, mu, alpha, a)
    tho = O.fit(x.astype(np.float64), y.astype(np.float64), m, W)
    assert rel(th, tho) <= 1e-5


@pytest.mark.parametrize("d,m", [(1, 40), (2, 10)])
def test_penalty_weights_match_oracle(d, m):
    lams = [1e-3, 2.5]
    W = host(fk.fk_penalty_weights(d, m, lams, s=1.5, mu=0.3, alpha=[[1] + [0] * (d - 1), [0] * (d - 1) + [2]],
                                   a=[1.0, -0.1]))
    for i, lam in enumerate(lams):
        want = O.penalty_pik(d, m, lam, 1.5, 0.3, [[1] + [0] * (d - 1), [0] * (d - 1) + [2]], [1.0, -0.1])
        assert np.max(np.abs(W[i] - want) / want) < 1e-14
    Wl = host(fk.fk_penalty_weights(d, m, [0.7], penalty=fk.FK_PEN_LOWBIAS))
    assert np.all(Wl == 0.7)


@pytest.mark.parametrize("d,m", [(1, 30), (2, 8)])
def test_cholesky_and_cg_agree_with_oracle_solve(d, m):
    x = S.uniform_points(5000, d, 27)
    To = O.moments(x, m)
    D = (2 * m + 1) ** d
    g = np.random.default_rng(7)
    rhs = g.standard_normal((3, D)) + 1j * g.standard_normal((3, D))
    lams = [1e-6, 1e-2]
    Wo = np.stack([O.penalty_sobolev(d, m, l, 1.0) for l in lams])
    T = torch.from_numpy(To).cuda()
    W = torch.from_numpy(Wo).cuda()
    R = torch.from_numpy(rhs).cuda()
    sol_c = host(fk.fk_solve(T, W, R, d, m, opts=fk.default_opts(solver=fk.FK_SOLVER_CHOL)))
    sol_g, rep = fk.fk_solve(T, W, R, d, m, opts=fk.default_opts(solver=fk.FK_SOLVER_CG), report=True)
    sol_g = host(sol_g)
    A = O.toeplitz_matrix(To, d, m)
    for li in range(2):
        want = O.solve_hpd(A + np.diag(Wo[li]), rhs.T).T
        assert rel(sol_c[li], want) < 1e-11
        assert rel(sol_g[li], want) < 1e-10
    assert rep["cg_iters"] > 0


@pytest.mark.parametrize("m", [15, 16])
def test_cg_corner_lags(m):
    # A shifted lattice of 2m points per period puts |T| at the lags +-2m on the order
    # of T_0, with T_(-2m) != T_(2m).  For m = 16 the cooperative CG's circulant has
    # length 4m and adds the lag -2m terms itself; m = 15 takes length 8m - 2 -> 64.
    lat = S.equispaced_2d(2 * m, 2 * m) + 0.3 / m
    x = np.concatenate([lat, S.uniform_points(3000, 2, 29)], axis=1)
    x = (x + np.pi) % (2 * np.pi) - np.pi
    To = O.moments(x, m)
    K2 = 4 * m + 1
    Tm = To.reshape(K2, K2)
    assert abs(Tm[0, 2 * m] - Tm[4 * m, 2 * m]) > 0.1 * Tm[2 * m, 2 * m].real
    D = (2 * m + 1) ** 2
    g = np.random.default_rng(8)
    rhs = g.standard_normal((2, D)) + 1j * g.standard_normal((2, D))
    lams = [1e-4, 1e-1]
    Wo = np.stack([O.penalty_sobolev(2, m, l, 1.5) for l in lams])
    sol = host(fk.fk_solve(torch.from_numpy(To).cuda(), torch.from_numpy(Wo).cuda(), torch.from_numpy(rhs).cuda(), 2,
                           m, opts=fk.default_opts(solver=fk.FK_SOLVER_CG, cg_tol=1e-13)))
    A = O.toeplitz_matrix(To, 2, m)
    for li in range(2):
        want = O.solve_hpd(A + np.diag(Wo[li]), rhs.T).T
        assert rel(sol[li], want) < 1e-10, li


@pytest.mark.parametrize("d", [1, 2])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_constant_mode_only(d, precision):
    # m = 0, the degenerate case: one mode, T_0 = 1 and W_0 = lambda (1 + 0^(2s)), so
    # theta_0 = mean(y) / (1 + lambda) and the prediction is that constant everywhere
    n, lam = 5001, 0.3
    td = torch.float32 if precision == "mixed" else torch.float64
    eps, tol = (1e-6, 1e-5) if precision == "mixed" else (1e-12, 1e-11)
    x = S.uniform_points(n, d, 41)
    y = 1.5 + np.sin(x[0])
    xs = x.astype(np.float32) if precision == "mixed" else x
    ys = y.astype(np.float32) if precision == "mixed" else y
    th = fk.fk_fit_sobolev(dev(xs, td), dev(ys, td), 0, 2.0, [lam], eps, precision)
    want = ys.astype(np.float64).mean() / (1.0 + lam)
    got = host(th)[0, 0]
    assert got.shape == (1,)
    assert abs(got[0] - want) < tol * abs(want)
    xq = S.uniform_points(300, d, 42)
    xq = xq.astype(np.float32) if precision == "mixed" else xq
    f = host(fk.fk_predict(th[0], dev(xq, td), 0, eps, precision))[0]
    assert np.max(np.abs(f - want)) < tol * abs(want)


def test_not_positive_definite_reported():
    m = 4
    x = S.uniform_points(100, 1, 28)
    T = torch.from_numpy(O.moments(x, m)).cuda()
    W = torch.full((1, 2 * m + 1), -5.0, dtype=torch.float64, device="cuda")
    R = torch.ones((1, 2 * m + 1), dtype=torch.complex128, device="cuda")
    with pytest.raises(fk.FkError) as e:
        fk.fk_solve(T, W, R, 1, m, opts=fk.default_opts(solver=fk.FK_SOLVER_CHOL))
    assert e.value.name == "FK_ENOTPD"


def test_points_out_of_range_reported():
    x = np.array([[0.1, 2.0, 12.0]], dtype=np.float32)
    c = np.ones(3, dtype=np.float32)
    with pytest.raises(fk.FkError) as e:
        fk.fk_type1(dev(x, torch.float32), dev(c, torch.float32), 4, 1e-6, "mixed")
    assert e.value.name == "FK_ERANGE"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_edge_points_fold_and_single_point(precision):
    td, nd = PREC[precision]
    # points at the period ends and beyond pi (folded), plus a lone point
    x = np.array([[-np.pi, np.pi - 1e-7, 3.0 * np.pi - 0.5, -3.0 * np.pi + 0.25, 0.0]]).astype(nd)
    c = np.array([1.0, -2.0, 0.5, 3.0, 1.5]).astype(nd)
    kmax = 6
    eps = 1e-12 if precision == "fp64" else 1e-6
    got = host(fk.fk_type1(dev(x, td), dev(c, td), kmax, eps, precision))[0]
    want = O.type1(x.astype(np.float64), c.astype(np.float64), kmax)
    assert rel(got, want) <= 10 * eps
    got1 = host(fk.fk_type1(dev(x[:, :1], td), dev(c[:1], td), kmax, eps, precision))[0]
    assert rel(got1, O.type1(x[:, :1].astype(np.float64), c[:1].astype(np.float64), kmax)) <= 10 * eps


def test_noiseless_recovery_is_exact_to_solve_precision():
    m = 10
    x = S.uniform_points(20000, 1, 29)
    y = S.bandlimited_1d(x)
    th = host(fk.fk_fit_sobolev(dev(x, torch.float64), dev(y, torch.float64), m, 1.0, [1e-13], 1e-12, "fp64",
                                penalty=fk.FK_PEN_LOWBIAS))[0, 0]
    assert abs(th[m + 3] - (-0.5j)) < 1e-10
    assert abs(th[m + 7] - 0.25) < 1e-10
    other = np.delete(th, [m - 7, m - 3, m + 3, m + 7])
    assert np.max(np.abs(other)) < 1e-10


# ---------------------------------------------------------------- binned register-accumulating spreader
@pytest.mark.parametrize("n", [1, 37, 5000, 1_300_001, 3_000_017])
def test_binned_spreader_matches_oracle(n):
    m, eps = 8, 1e-6
    x, y = S.wl2_sobolev_2d(n, dtype=np.float32)
    opts = fk.default_opts(spread=fk.FK_SPREAD_BINNED)
    T, b = fk.fk_build_system(dev(x, torch.float32), dev(y, torch.float32), m, eps, "mixed", opts=opts)
    To = O.moments(x.astype(np.float64), m)
    bo = O.rhs(x.astype(np.float64), y.astype(np.float64), m)
    assert rel(host(T), To) <= 10 * eps
    assert rel(host(b)[0], bo) <= 10 * eps


def test_binned_and_atomic_spreaders_agree_config2_grid():
    # the workload's grid (m = 32: 129 x 129 moments, N = 256, w = 7) over several chunks
    m, eps = 32, 1e-6
    x, y = S.wl2_sobolev_2d(4_000_037, dtype=np.float32)
    xd, yd = dev(x, torch.float32), dev(y, torch.float32)
    Tb, bb = fk.fk_build_system(xd, yd, m, eps, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_BINNED))
    Ta, ba = fk.fk_build_system(xd, yd, m, eps, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_ATOMIC))
    assert rel(host(Tb), host(Ta)) < 1e-6
    assert rel(host(bb), host(ba)) < 1e-6
    # sampled moments against direct sums over all points
    j = [(0, 1), (5, -7), (-64, 64), (33, 2)]
    K = 4 * m + 1
    Tg = host(Tb)
    for j0, j1 in j:
        want = np.mean(np.exp(-1j * (j0 * x[0].astype(np.float64) + j1 * x[1].astype(np.float64))))
        assert abs(Tg[(j0 + 2 * m) * K + (j1 + 2 * m)] - want) < 1e-6


def test_binned_clustered_points_two_owner_sizes():
    # the workload's grid (N = 256: owners of 256 cells, then of 192) with crowded
    # points, which overflow the one-pass buckets: the exact partition, with the same
    # owner map, takes over on the device
    m, eps, n = 32, 1e-6, 1_500_001
    g = np.random.default_rng(97)
    x = np.clip(g.normal(-0.8, 0.03, size=(2, n)), -np.pi, np.pi - 1e-6).astype(np.float32)
    x[:, : n // 5] = S.uniform_points(n // 5, 2, 36).astype(np.float32)
    y = np.sin(x[1].astype(np.float64)).astype(np.float32)
    xd, yd = dev(x, torch.float32), dev(y, torch.float32)
    Tb, bb = fk.fk_build_system(xd, yd, m, eps, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_BINNED))
    Ta, ba = fk.fk_build_system(xd, yd, m, eps, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_ATOMIC))
    assert rel(host(Tb), host(Ta)) < 1e-6
    assert rel(host(bb), host(ba)) < 1e-6
    K = 4 * m + 1
    Tg = host(Tb)
    x0, x1 = x[0].astype(np.float64), x[1].astype(np.float64)
    for j0, j1 in [(0, 0), (3, -1), (-64, 64), (17, 40)]:
        want = np.mean(np.exp(-1j * (j0 * x0 + j1 * x1)))
        assert abs(Tg[(j0 + 2 * m) * K + (j1 + 2 * m)] - want) < 1e-6


def test_binned_rejects_out_of_range_points():
    x = S.uniform_points(2000, 2, 32).astype(np.float32)
    x[1, 1234] = 20.0
    c = np.ones(2000, dtype=np.float32)
    with pytest.raises(fk.FkError) as e:
        fk.fk_build_system(dev(x, torch.float32), dev(c, torch.float32), 4, 1e-6, "mixed",
                           opts=fk.default_opts(spread=fk.FK_SPREAD_BINNED))
    assert e.value.name == "FK_ERANGE"


@pytest.mark.parametrize("n", [200_000, 1_000_003])
def test_binned_spreader_clustered_points(n):
    # points crowded into a few cells overflow the one-pass partition's buckets; the
    # exact count-scan-scatter partition then takes over on the device
    m, eps = 16, 1e-6
    g = np.random.default_rng(99)
    x = np.clip(g.normal(0.3, 0.02, size=(2, n)), -np.pi, np.pi - 1e-6).astype(np.float32)
    x[:, : n // 10] = S.uniform_points(n // 10, 2, 33).astype(np.float32)  # and a uniform tenth
    y = np.cos(x[0].astype(np.float64)).astype(np.float32)
    T, b = fk.fk_build_system(dev(x, torch.float32), dev(y, torch.float32), m, eps, "mixed",
                              opts=fk.default_opts(spread=fk.FK_SPREAD_BINNED))
    To = O.moments(x.astype(np.float64), m)
    bo = O.rhs(x.astype(np.float64), y.astype(np.float64), m)
    assert rel(host(T), To) <= 10 * eps
    assert rel(host(b)[0], bo) <= 10 * eps


@pytest.mark.parametrize("with_y", [True, False])
def test_binned_all_points_in_one_cell(with_y):
    # every point at the same place: each accumulation round finds one cell holding all
    # of its records, far past the cell's slots, so most records move to the next round
    # or go straight into the grid; the normalised sums are e^{-i j x} (b: times the
    # mean strength)
    m, eps, n = 12, 1e-6, 150_001
    x0 = np.array([0.7312, -2.0419], dtype=np.float32)
    x = np.repeat(x0[:, None], n, axis=1)
    y = np.linspace(0.5, 1.5, n).astype(np.float32) if with_y else None
    T, b = fk.fk_build_system(dev(x, torch.float32), dev(y, torch.float32) if with_y else None, m, eps, "mixed",
                              opts=fk.default_opts(spread=fk.FK_SPREAD_BINNED))
    xs = x0.astype(np.float64)
    j = np.arange(-2 * m, 2 * m + 1)
    To = np.exp(-1j * (j[:, None] * xs[0] + j[None, :] * xs[1])).ravel()
    assert rel(host(T), To) <= 10 * eps
    if with_y:
        k = np.arange(-m, m + 1)
        bo = np.exp(-1j * (k[:, None] * xs[0] + k[None, :] * xs[1])).ravel() * np.mean(y.astype(np.float64))
        assert rel(host(b)[0], bo) <= 10 * eps


@pytest.mark.parametrize("kind", ["uniform", "ragged", "clustered"])
def test_binned_moments_ones_only(kind):
    # moments alone (no strengths): the one-pass partition writes 8-byte records; crowded
    # points fall back to the exact partition's 16-byte records
    m, eps = 16, 1e-6
    if kind == "clustered":
        n = 300_000
        g = np.random.default_rng(98)
        x = np.clip(g.normal(-1.1, 0.02, size=(2, n)), -np.pi, np.pi - 1e-6).astype(np.float32)
        x[:, : n // 10] = S.uniform_points(n // 10, 2, 34).astype(np.float32)
    else:
        n = 1_000_000 if kind == "uniform" else 1_000_003
        x = S.uniform_points(n, 2, 35).astype(np.float32)
    T, b = fk.fk_build_system(dev(x, torch.float32), None, m, eps, "mixed",
                              opts=fk.default_opts(spread=fk.FK_SPREAD_BINNED))
    assert rel(host(T), O.moments(x.astype(np.float64), m)) <= 10 * eps


@pytest.mark.parametrize("d,m,solver", [(1, 30, "cg"), (2, 10, "chol"), (2, 12, "cg")])
def test_sobolev_pairs_sweep(d, m, solver):
    # 6 (s, lambda) pairs from one spreading pass, each against its own oracle fit
    n = 8000
    x = S.uniform_points(n, d, 61)
    y = (np.sin(x[0]) * (np.cos(x[1]) if d == 2 else 1.0) + 0.1 * np.random.default_rng(4).standard_normal(n))
    pairs = [(0.5, 1e-3), (1.0, 1e-3), (1.5, 1e-4), (2.0, 1e-5), (2.5, 1e-2), (1.25, 3e-4)]
    opts = fk.default_opts(solver=fk.FK_SOLVER_CHOL if solver == "chol" else fk.FK_SOLVER_CG, cg_tol=1e-13)
    th = fk.fk_fit_sobolev_pairs(dev(x, torch.float64), dev(y, torch.float64), m, [p[0] for p in pairs],
                                 [p[1] for p in pairs], 1e-12, "fp64", opts=opts).cpu().numpy()
    for i, (s, lam) in enumerate(pairs):
        want = O.fit(x, y, m, O.penalty_sobolev(d, m, lam, s))
        assert rel(th[i, 0], want) < 1e-9, (s, lam)


@pytest.mark.parametrize("kmax,eps", [(30, 1e-6), (13, 1e-3), (3, 1e-6)])
def test_type2_shared_grid_path_matches_direct_sums(kmax, eps):
    # mixed 2-D type-2 on fine grids of <= 128^2 nodes (here 128^2 and 16^2 at width 7,
    # 64^2 at width 4) interpolates from a copy of the grid in shared memory: several
    # coefficient sets, a ragged n, and points at the ends of [-3 pi, 3 pi) whose windows
    # wrap (on the 16-node grid a 7-wide window wraps for most points)
    n = 20_003
    x = S.uniform_points(n, 2, 24)
    x[:, :64] = np.float32(-3 * np.pi) + np.float32(1e-6)
    x[:, 64:128] = np.nextafter(np.float32(3 * np.pi), np.float32(0)) - np.float32(1e-6)
    x[:, 128:192] = np.float32(np.pi)
    x = x.astype(np.float32)
    g = np.random.default_rng(7)
    D = (2 * kmax + 1) ** 2
    coef = g.standard_normal((3, D)) + 1j * g.standard_normal((3, D))
    got = host(fk.fk_type2(torch.from_numpy(coef).cuda(), dev(x, torch.float32), kmax, eps, "mixed"))
    for s_ in range(3):
        want = O.type2(coef[s_], x.astype(np.float64), kmax)
        assert rel(got[s_], want.real) <= 10 * eps * np.linalg.norm(want) / np.linalg.norm(want.real)
