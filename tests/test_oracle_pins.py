"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
brute-force kernel ridge regression, discrete orthogonality, invariants, tiny
scalar loops and finite differences.  None of these needs a GPU.
"""
import cmath
import json
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "bandlimited_coeffs.json")))


def _coef_vec(table: dict, d: int, m: int) -> np.ndarray:
    K = 2 * m + 1
    th = np.zeros((K,) * d, dtype=np.complex128)
    for key, val in table.items():
        if key.startswith("_"):
            continue
        idx = tuple(int(v) + m for v in key.split(","))
        th[idx] = val[0] + 1j * val[1]
    return th.ravel()


def _idx(d, m, k):
    """Flat index of mode k in the lexicographic grid (last dimension fastest)."""
    K = 2 * m + 1
    f = 0
    for l in range(d):
        f = f * K + (k[l] + m)
    return f


# ----------------------------------------------------------------- type-1 / type-2
def test_type1_matches_scalar_loop():
    rng = np.random.default_rng(1)
    for d, kmax in [(1, 3), (2, 2), (3, 1)]:
        x = rng.uniform(-np.pi, np.pi, (d, 7))
        c = rng.standard_normal(7) + 0.3j * rng.standard_normal(7)
        got = O.type1(x, c, kmax)
        ks = O.mode_grid(d, kmax)
        want = np.array([sum(c[i] * cmath.exp(-1j * sum(k[l] * x[l, i] for l in range(d)))
                             for i in range(7)) for k in ks])
        assert np.max(np.abs(got - want)) < 1e-13


def test_type2_matches_scalar_loop():
    rng = np.random.default_rng(2)
    for d, kmax in [(1, 3), (2, 2), (3, 1)]:
        ks = O.mode_grid(d, kmax)
        coef = rng.standard_normal(len(ks)) + 1j * rng.standard_normal(len(ks))
        x = rng.uniform(-np.pi, np.pi, (d, 5))
        got = O.type2(coef, x, kmax)
        want = np.array([sum(coef[t] * cmath.exp(1j * sum(ks[t][l] * x[l, i] for l in range(d)))
                             for t in range(len(ks))) for i in range(5)])
        assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("d,kmax", [(1, 9), (2, 4), (3, 2)])
def test_type1_type2_adjoint(d, kmax):
    rng = np.random.default_rng(3)
    n = 300
    x = rng.uniform(-np.pi, np.pi, (d, n))
    c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    D = (2 * kmax + 1) ** d
    th = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    lhs = np.vdot(O.type1(x, c, kmax), th)
    rhs = np.vdot(c, O.type2(th, x, kmax))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_mode_grid_order():
    k = O.mode_grid(2, 1)
    assert k.tolist() == [[-1, -1], [-1, 0], [-1, 1], [0, -1], [0, 0], [0, 1], [1, -1], [1, 0], [1, 1]]


# ----------------------------------------------------------------- moments
def test_equispaced_moments_are_kronecker_delta_1d():
    # discrete orthogonality: (1/n) sum_i e^{-i j X_i} = [j == 0 mod n] on X_i = -pi + 2 pi i/n
    m, n = 10, 64
    T = O.moments(S.equispaced_1d(n), m)
    want = np.zeros(4 * m + 1)
    want[2 * m] = 1.0
    assert np.max(np.abs(T - want)) < 1e-14


def test_equispaced_moments_are_kronecker_delta_2d():
    m = 4
    T = O.moments(S.equispaced_2d(20, 23), m).reshape(4 * m + 1, 4 * m + 1)
    want = np.zeros_like(T)
    want[2 * m, 2 * m] = 1.0
    assert np.max(np.abs(T - want)) < 1e-14


@pytest.mark.parametrize("d,m", [(1, 12), (2, 4)])
def test_toeplitz_invariants(d, m):
    x = S.uniform_points(500, d, 11)
    T = O.moments(x, m)
    K2 = 4 * m + 1
    c = _idx(d, 2 * m, (0,) * d)
    assert abs(T[c] - 1.0) < 1e-15                       # T_0 = n/n
    Tg = T.reshape((K2,) * d)
    flip = Tg[(slice(None, None, -1),) * d]
    assert np.max(np.abs(flip - np.conj(Tg))) < 1e-14     # T_{-j} = conj(T_j)
    assert np.max(np.abs(T)) <= 1.0 + 1e-14               # |T_j| <= 1
    A = O.toeplitz_matrix(T, d, m)
    assert np.max(np.abs(A - A.conj().T)) < 1e-15         # Hermitian
    assert np.linalg.eigvalsh(A).min() > -1e-12           # Phi^*Phi/n is PSD


@pytest.mark.parametrize("d", [1, 2])
def test_rhs_equals_toeplitz_times_coefficients(d):
    # Y = f*(X) band-limited at |k| <= m0 <= m:  b = Toep(T) theta*  exactly, any points
    m = 8
    x = S.uniform_points(700, d, 12)
    f = S.bandlimited_1d if d == 1 else S.bandlimited_2d
    th = _coef_vec(GOLD["bandlimited_%dd" % d], d, m)
    b = O.rhs(x, f(x), m)
    A = O.toeplitz_matrix(O.moments(x, m), d, m)
    assert np.max(np.abs(b - A @ th)) < 1e-13


# ----------------------------------------------------------------- closed forms of the fit
def test_equispaced_sobolev_closed_form_1d():
    # T = I and b = theta*, so theta_hat_k = theta*_k / (1 + lambda (1 + |k|^{2s}))  (Prop. 3.1)
    m, lam, s = 12, 0.3, 1.5
    x = S.equispaced_1d(64)
    th = O.fit(x, S.bandlimited_1d(x), m, O.penalty_sobolev(1, m, lam, s))
    star = _coef_vec(GOLD["bandlimited_1d"], 1, m)
    k = np.arange(-m, m + 1)
    want = star / (1.0 + lam * (1.0 + np.abs(k) ** (2 * s)))
    assert np.max(np.abs(th - want)) < 1e-14


def test_equispaced_lowbias_closed_form_2d():
    m, lam = 6, 0.25
    x = S.equispaced_2d(26, 27)
    th = O.fit(x, S.bandlimited_2d(x), m, O.penalty_lowbias(2, m, lam))
    star = _coef_vec(GOLD["bandlimited_2d"], 2, m)
    assert np.max(np.abs(th - star / (1.0 + lam))) < 1e-14


def test_heat_operator_symbol_and_pik_closed_form():
    m, lam, s, mu = 6, 1e-3, 1.0, 0.5
    alpha = [[1, 0], [0, 2]]
    a = [1.0, -0.1]                   # P = d_t - 0.1 d_xx, coordinate 0 is t
    P2 = np.abs(O.pde_symbol(2, m, alpha, a)) ** 2
    for (kt, kx), val in GOLD["heat_symbol"]["samples"]:
        assert abs(P2[_idx(2, m, (kt, kx))] - val) < 1e-12
    x = S.equispaced_2d(26, 26)
    W = O.penalty_pik(2, m, lam, s, mu, alpha, a)
    th = O.fit(x, S.bandlimited_2d(x), m, W)
    k = O.mode_grid(2, m)
    sob = lam * (1.0 + (k[:, 0] ** 2 + k[:, 1] ** 2) ** s)
    heat = k[:, 0] ** 2 + 0.01 * k[:, 1] ** 4
    star = _coef_vec(GOLD["bandlimited_2d"], 2, m)
    assert np.max(np.abs(th - star / (1.0 + sob + mu * heat))) < 1e-14


def test_sobolev_weight_zero_mode_and_fractional_s():
    W = O.penalty_sobolev(2, 2, 2.0, 0.75, c0=1.0)
    k = O.mode_grid(2, 2)
    r = np.sqrt(k[:, 0] ** 2 + k[:, 1] ** 2)
    assert np.allclose(W, 2.0 * (1.0 + r ** 1.5), rtol=1e-15, atol=0)
    assert W[_idx(2, 2, (0, 0))] == 2.0


def test_noiseless_recovery_sign_convention():
    # random points, Y = sin(3X) + 0.5cos(7X): theta_hat -> theta* as lambda -> 0,
    # in particular theta_3 = -i/2 (fixes the e^{-ikX} sign of b, Q1)
    m = 10
    x = S.uniform_points(3000, 1, 13)
    th = O.fit(x, S.bandlimited_1d(x), m, O.penalty_lowbias(1, m, 1e-12))
    star = _coef_vec(GOLD["bandlimited_1d"], 1, m)
    assert np.max(np.abs(th - star)) < 1e-9
    assert abs(th[m + 3] - (-0.5j)) < 1e-9
    xq = S.uniform_points(50, 1, 14)
    assert np.max(np.abs(O.predict(th, xq, m) - S.bandlimited_1d(xq))) < 1e-8
    assert np.max(np.abs(O.predict_imag(th, xq, m))) < 1e-12


# ----------------------------------------------------------------- brute-force KRR (§2.1)
def test_krr_bruteforce_1d_matches_fourier_fit():
    m, lam, s = 50, 1e-4, 1.0
    x, y = S.wl1_sobolev_1d(2000)
    W = O.penalty_sobolev(1, m, lam, s)
    xq = S.uniform_points(64, 1, 15)
    fq, th_krr = O.krr_bruteforce(x, y, m, W, xq)
    th = O.fit(x, y, m, W)
    assert np.linalg.norm(th - th_krr) / np.linalg.norm(th_krr) < 1e-11
    f = O.predict(th, xq, m)
    assert np.linalg.norm(f - fq) / np.linalg.norm(fq) < 1e-11


def test_krr_bruteforce_2d_matches_fourier_fit():
    m, lam, s = 3, 1e-3, 2.0
    x, y = S.wl2_sobolev_2d(400, dtype=np.float64)
    W = O.penalty_sobolev(2, m, lam, s)
    xq = S.uniform_points(40, 2, 16)
    fq, th_krr = O.krr_bruteforce(x, y, m, W, xq)
    th = O.fit(x, y, m, W)
    assert np.linalg.norm(th - th_krr) / np.linalg.norm(th_krr) < 1e-11
    assert np.linalg.norm(O.predict(th, xq, m) - fq) / np.linalg.norm(fq) < 1e-11


# ----------------------------------------------------------------- additive model (§5)
def test_additive_blocks():
    d, m, n = 3, 4, 600
    X = S.uniform_points(n, d, 17)
    G = O.additive_gram(X, m)
    K = 2 * m + 1
    assert np.max(np.abs(G - G.conj().T)) < 1e-15
    for l1 in range(d):
        # diagonal block: Toeplitz from the 1-D moments of coordinate l1
        Tl = O.moments(X[l1:l1 + 1], m)
        assert np.max(np.abs(G[l1 * K:(l1 + 1) * K, l1 * K:(l1 + 1) * K]
                             - O.toeplitz_matrix(Tl, 1, m))) < 1e-14
        for l2 in range(d):
            B = G[l1 * K:(l1 + 1) * K, l2 * K:(l2 + 1) * K]
            assert abs(B[m, m] - 1.0) < 1e-14
            # column k2 = 0: the 1-D moments of coordinate l1 over |k1| <= m
            assert np.max(np.abs(B[:, m] - Tl[m:3 * m + 1])) < 1e-14
            if l1 != l2:
                # a 2-D type-1 transform of ones at (X_l1, -X_l2)  (§5, Complexity)
                pts = np.stack([X[l1], -X[l2]])
                assert np.max(np.abs(B.ravel() - O.type1(pts, np.ones(n), m) / n)) < 1e-14


def test_additive_fit_matches_krr():
    d, m, lam = 3, 3, 1e-3
    X, y = S.wl4_additive(500, d=d, dtype=np.float64)
    th = O.fit_additive(X, y, m, lam)
    Xq = S.uniform_points(30, d, 18)
    fq = O.additive_krr(X, y, m, lam, Xq)
    assert np.linalg.norm(O.predict_additive(th, Xq, m) - fq) / np.linalg.norm(fq) < 1e-10
    # the d intercepts are equal (the k = 0 columns coincide, Q10)
    K = 2 * m + 1
    ic = th.reshape(d, K)[:, m]
    assert np.max(np.abs(ic - ic[0])) < 1e-10


# ----------------------------------------------------------------- hypergradient vs FD
def test_hypergradient_matches_finite_differences():
    d, m = 2, 4
    lam, s, mu = 1e-2, 1.0, 3e-2
    alpha, a = [[1, 0], [0, 2]], [1.0, -0.1]
    x, y = S.wl3_pik_heat(900, dtype=np.float64)
    xv, yv = S.wl3_pik_heat(300, dtype=np.float64, validation=True)

    def loss(lam_, s_, mu_, a_, y_=y):
        W = O.penalty_pik(d, m, lam_, s_, mu_, alpha, a_)
        return O.heldout_loss(O.fit(x, y_, m, W), xv, yv, m)

    W = O.penalty_pik(d, m, lam, s, mu, alpha, a)
    L, th, dW, dY = O.hypergradient(x, y, xv, yv, m, W)
    assert abs(L - loss(lam, s, mu, a)) < 1e-14
    g = O.penalty_param_grads(d, m, lam, s, mu, alpha, a, dW)

    def fd(f, v, rel=1e-5):
        h = rel * max(abs(v), 1e-3)
        return (f(v + h) - f(v - h)) / (2 * h)

    assert abs(fd(lambda v: loss(v, s, mu, a), lam) - g["lambda"]) < 1e-6 * abs(g["lambda"]) + 1e-12
    assert abs(fd(lambda v: loss(lam, v, mu, a), s) - g["s"]) < 1e-6 * abs(g["s"]) + 1e-12
    assert abs(fd(lambda v: loss(lam, s, v, a), mu) - g["mu"]) < 1e-6 * abs(g["mu"]) + 1e-12
    ga = fd(lambda v: loss(lam, s, mu, [a[0], v]), a[1])
    assert abs(ga - g["a"][1]) < 1e-6 * abs(g["a"][1]) + 1e-12
    for i in [0, 17, 401]:
        def ly(v, i=i):
            yy = y.copy()
            yy[i] = v
            return loss(lam, s, mu, a, yy)
        assert abs(fd(ly, y[i], rel=1e-3) - dY[i]) < 1e-6 * abs(dY[i]) + 1e-12


# ------------------------------------------------------------------ sub-domain / collocation PIK
def test_box_moments_full_period_is_identity():
    for d in (1, 2):
        c = O.box_moments(d, 3, -np.pi, np.pi)
        want = np.zeros_like(c)
        want[len(c) // 2] = 1.0
        assert np.max(np.abs(c - want)) < 1e-15


def test_box_moments_against_quadrature():
    # midpoint rule on a fine grid of the box (exact for these smooth integrands up to
    # O(h^2 j^2))
    lo, hi, m = (-0.3, 0.1), (0.9, 1.2), 3
    c = O.box_moments(2, m, lo, hi)
    K = 4 * m + 1
    g = 4000
    u = lo[0] + (hi[0] - lo[0]) * (np.arange(g) + 0.5) / g
    v = lo[1] + (hi[1] - lo[1]) * (np.arange(g) + 0.5) / g
    area = (hi[0] - lo[0]) * (hi[1] - lo[1]) / g ** 2
    for j0, j1 in [(0, 0), (1, -2), (-5, 3), (6, 6)]:
        q = np.sum(np.exp(-1j * j0 * u))[()] * np.sum(np.exp(-1j * j1 * v)) * area / (2 * np.pi) ** 2
        assert abs(c[(j0 + 2 * m) * K + (j1 + 2 * m)] - q) < 1e-6


def test_penalty_form_is_the_integral_of_the_operator():
    # theta^* (D^* C D) theta = (2 pi)^{-d} int_Omega |D f_theta|^2 dx, by quadrature of
    # D f_theta built from its definition (derivatives of e^{i<k,x>})
    g = np.random.default_rng(5)
    m, lo, hi = 4, (-0.7, 0.2), (0.8, 1.5)
    alpha, a = [[1, 0], [0, 2]], [1.0, -0.3]
    D = (2 * m + 1) ** 2
    th = g.standard_normal(D) + 1j * g.standard_normal(D)
    Pen = O.penalty_pik_general(2, m, 0.0, 1.0, 1.0, alpha, a, O.box_moments(2, m, lo, hi))
    form = np.real(np.conj(th) @ Pen @ th)
    k = O.mode_grid(2, m).astype(np.float64)
    npt = 600
    u = lo[0] + (hi[0] - lo[0]) * (np.arange(npt) + 0.5) / npt
    v = lo[1] + (hi[1] - lo[1]) * (np.arange(npt) + 0.5) / npt
    U, V = np.meshgrid(u, v, indexing="ij")
    Df = np.zeros(U.shape, dtype=np.complex128)
    for t, (al, coef) in enumerate(zip(alpha, a)):
        # d^al / dx^al of e^{i(k0 u + k1 v)} = (i k0)^al0 (i k1)^al1 e^{...}
        fac = coef * (1j * k[:, 0]) ** al[0] * (1j * k[:, 1]) ** al[1]
        Df += np.einsum("k,kij->ij", th * fac, np.exp(1j * (k[:, 0, None, None] * U + k[:, 1, None, None] * V)))
    integral = np.sum(np.abs(Df) ** 2) * (hi[0] - lo[0]) * (hi[1] - lo[1]) / npt ** 2 / (2 * np.pi) ** 2
    assert abs(form - integral) < 1e-5 * abs(integral)


def test_collocation_moments_full_period_match_the_diagonal_penalty():
    # equispaced collocation points over the period: their moments are delta_j, so the
    # collocation penalty equals the full-period (diagonal) one
    m = 3
    xr = S.equispaced_2d(16, 16)
    c = O.moments(xr, m)
    Pen = O.penalty_pik_general(2, m, 1e-3, 1.0, 0.5, [[1, 0], [0, 2]], [1.0, -0.1], c)
    want = np.diag(O.penalty_pik(2, m, 1e-3, 1.0, 0.5, [[1, 0], [0, 2]], [1.0, -0.1]))
    assert np.max(np.abs(Pen - want)) < 1e-12 * np.max(np.abs(want))


def test_general_pik_fit_minimises_the_objective():
    # the fit zeroes the gradient of n^-1 |Phi theta - Y|^2 + theta^* Pen theta, checked
    # with the objective evaluated by direct sums and finite differences along random
    # directions
    g = np.random.default_rng(8)
    m, n = 3, 400
    x = S.uniform_points(n, 2, 41)
    y = np.sin(x[0]) * np.cos(x[1]) + 0.1 * g.standard_normal(n)
    Pen = O.penalty_pik_general(2, m, 1e-2, 1.0, 0.3, [[1, 0], [0, 2]], [1.0, -0.1],
                                O.box_moments(2, m, (-1.0, -0.5), (1.2, 0.9)))
    th = O.fit_penalised(x, y, m, Pen)

    def objective(t):
        r = O.type2(t, x, m) - y  # complex predictions; the real target
        return float(np.mean(np.abs(r) ** 2) + np.real(np.conj(t) @ Pen @ t))

    J0 = objective(th)
    for _ in range(4):
        dirn = g.standard_normal(th.shape) + 1j * g.standard_normal(th.shape)
        h = 1e-4
        assert objective(th + h * dirn) - J0 > -1e-12
        assert objective(th - h * dirn) - J0 > -1e-12
        # second-order: the first-order term vanishes
        fd = (objective(th + h * dirn) - objective(th - h * dirn)) / (2 * h)
        assert abs(fd) < 1e-6
