"""The 1-D sweep at scale: counter-based generation on the device, fixed-point
spreading of many channels, streaming accumulation over chunks, and the batched
solve over 256 lambdas x 16 targets.

Tolerances: NUFFT pieces <= 10 eps normwise against the oracle; fits <= 1e-5
normwise per (lambda, target) on the mixed path; generated X bit for bit, Y to a few
fp32 ulps (CUDA's fp32 libm against the host twin's fp64-rounded steps).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

fk = pytest.importorskip("paper_2509_02649_b300")

M_SWEEP = 1000
LAMBDAS = np.logspace(-12, -2, 256)


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def host(t):
    return t.detach().cpu().numpy()


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("first,n", [(0, 1_000_003), ((1 << 34) + 8, 4099)])
def test_generator_matches_host_twin(first, n):
    x, y, amax = fk.generate_sweep_1d(first, n, 16)
    torch.cuda.synchronize()
    xh, yh = S.sweep_counter_points(first, n, 16)
    assert np.array_equal(host(x)[0], xh)
    yd = host(y)
    err = np.abs(yd.astype(np.float64) - yh.astype(np.float64))
    assert np.max(err / np.maximum(1.0, np.abs(yh))) < 2e-6
    # max |Y_t| of the chunk, as written by the generator
    want = np.abs(yd).max(axis=1).astype(np.float32).view(np.int32)
    assert np.array_equal(host(amax), want)


def sweep_sample(n, nt=16):
    x, y = S.sweep_counter_points(0, n, nt)
    return x[None, :], y


@pytest.mark.parametrize("n", [1, 37, 6001])
def test_fixed_spread_matches_oracle(n):
    x, y = sweep_sample(n)
    T, b = fk.fk_build_system(dev(x), dev(y), M_SWEEP, 1e-6, "mixed")
    To = O.moments(x.astype(np.float64), M_SWEEP)
    bo = O.rhs(x.astype(np.float64), y.astype(np.float64), M_SWEEP)
    assert rel(host(T), To) < 1e-5
    for t in range(16):
        assert rel(host(b)[t], bo[t]) < 1e-5


@pytest.mark.parametrize("eps", [1e-3, 1e-5])
def test_fixed_spread_other_widths(eps):
    x, y = sweep_sample(3001, 3)
    m = 40
    T, b = fk.fk_build_system(dev(x), dev(y), m, eps, "mixed")
    assert rel(host(T), O.moments(x.astype(np.float64), m)) < 10 * eps
    assert rel(host(b), O.rhs(x.astype(np.float64), y.astype(np.float64), m)) < 10 * eps


def test_fixed_spread_against_atomic_spread():
    x, y = sweep_sample(50_000)
    X, Y = dev(x), dev(y)
    Tf, bf = fk.fk_build_system(X, Y, M_SWEEP, 1e-6, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_FIXED))
    Ta, ba = fk.fk_build_system(X, Y, M_SWEEP, 1e-6, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_ATOMIC))
    assert rel(host(Tf), host(Ta)) < 1e-6
    assert rel(host(bf), host(ba)) < 1e-6


@pytest.mark.parametrize("m,nt,n", [(20, 2, 300_001), (50, 1, 1_000_000), (50, 4, 77_777), (100, 0, 2_000_003),
                                    (50, 1, 3)])
def test_fixed_spread_lane_copies_match_one_copy(m, nt, n):
    # grids of 256, 512 and 1024 nodes, where 32 lane copies fit in shared memory: the
    # integer sums are the same whichever copy each addition went to, so the moments
    # and right-hand sides agree bit for bit with the one-copy layout (ragged n takes the
    # scalar load path; the last case has a single CTA and three points)
    x, y = sweep_sample(n, max(nt, 1))
    X = dev(x)
    Y = dev(y[:nt]) if nt else None
    T1, b1 = fk.fk_build_system(X, Y, m, 1e-6, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_FIXED))
    T0, b0 = fk.fk_build_system(X, Y, m, 1e-6, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_FIXED_SHARED))
    assert torch.equal(T1, T0) and torch.equal(b1, b0)
    To = O.moments(x.astype(np.float64), m)
    assert rel(host(T1), To) < 1e-5


def test_fixed_spread_lane_copies_low_words_wrap():
    # every point at one node: each lane copy's low words wrap many times, and the
    # carries go to the shared high words; same sums as the one-copy layout
    n, m = 2_000_000, 50
    x = np.full((1, n), np.float32(-1.1), dtype=np.float32)
    y = (1.0 + 0.5 * np.random.default_rng(5).random((1, n))).astype(np.float32)
    X, Y = dev(x), dev(y)
    T1, b1 = fk.fk_build_system(X, Y, m, 1e-6, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_FIXED))
    T0, b0 = fk.fk_build_system(X, Y, m, 1e-6, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_FIXED_SHARED))
    assert torch.equal(T1, T0) and torch.equal(b1, b0)
    j = np.arange(-2 * m, 2 * m + 1)
    assert rel(host(T1), np.exp(-1j * j * np.float64(x[0, 0]))) < 1e-5


def test_fixed_spread_is_bitwise_reproducible():
    x, y = sweep_sample(200_000)
    X, Y = dev(x), dev(y)
    T1, b1 = fk.fk_build_system(X, Y, M_SWEEP, 1e-6, "mixed")
    T2, b2 = fk.fk_build_system(X, Y, M_SWEEP, 1e-6, "mixed")
    assert torch.equal(T1, T2) and torch.equal(b1, b2)


def test_fixed_spread_low_word_wraps():
    # 3e6 points at one position: every CTA adds thousands of same-sign contributions
    # to the same nodes, so the 32-bit low words wrap many times.  Closed form:
    # T_j = e^{-i j x0}, b_k = mean(y) e^{-i k x0}.
    n, m = 3_000_000, 20
    x0 = np.float32(0.3)
    x = np.full((1, n), x0, dtype=np.float32)
    y = (1.0 + 0.5 * np.random.default_rng(3).random((2, n))).astype(np.float32)
    T, b = fk.fk_build_system(dev(x), dev(y), m, 1e-6, "mixed", opts=fk.default_opts(spread=fk.FK_SPREAD_FIXED))
    j = np.arange(-2 * m, 2 * m + 1)
    assert rel(host(T), np.exp(-1j * j * np.float64(x0))) < 1e-5
    k = np.arange(-m, m + 1)
    for t in range(2):
        assert rel(host(b)[t], y[t].astype(np.float64).mean() * np.exp(-1j * k * np.float64(x0))) < 1e-5


def test_fixed_spread_scale_handling():
    x, y = sweep_sample(20_000, 3)
    X = dev(x)
    _, b = fk.fk_build_system(X, dev(y), 50, 1e-6, "mixed")
    # a power-of-two factor moves the fixed-point scale by the same power: exact
    _, b40 = fk.fk_build_system(X, dev(y * np.float32(2.0 ** 40)), 50, 1e-6, "mixed")
    assert torch.equal(b40, b * 2.0 ** 40)
    # tiny and zero channels
    y2 = np.stack([y[0] * np.float32(1e-30), np.zeros_like(y[0]), y[2]])
    _, b2 = fk.fk_build_system(X, dev(y2), 50, 1e-6, "mixed")
    bo = O.rhs(x.astype(np.float64), y2.astype(np.float64), 50)
    assert rel(host(b2)[0], bo[0]) < 1e-5
    assert torch.count_nonzero(b2[1]) == 0
    assert rel(host(b2)[2], bo[2]) < 1e-5


@pytest.mark.parametrize("d", [1, 2])
def test_accumulator_chunks(d):
    n = 6000
    if d == 1:
        x, y = sweep_sample(n, 2)
        m = 60
    else:
        x, y1 = S.wl2_sobolev_2d(n)
        y = y1[None, :]
        m = 12
    acc = fk.Accumulator(d, m, y.shape[0], 1e-6, "mixed")
    for a, b in [(0, 1000), (1000, 4003), (4003, n)]:
        acc.add(dev(x[:, a:b]), dev(y[:, a:b]))
    T, bb, ntot = acc.system()
    acc.close()
    assert ntot == n
    To = O.moments(x.astype(np.float64), m)
    bo = O.rhs(x.astype(np.float64), y.astype(np.float64), m)
    assert rel(host(T), To) < 1e-5
    assert rel(host(bb), bo) < 1e-5


def test_accumulator_range_error():
    x, y = sweep_sample(1000, 1)
    x = x.copy()
    x[0, 17] = 10.0
    acc = fk.Accumulator(1, 20, 1, 1e-6, "mixed")
    acc.add(dev(x), dev(y))
    with pytest.raises(fk.FkError) as e:
        acc.system()
    assert e.value.name == "FK_ERANGE"
    acc.close()


def test_sweep_small_sample_vs_oracle():
    n = 1 << 15
    x, y, amax = fk.generate_sweep_1d(0, n, 16)
    xh, yh = S.sweep_counter_points(0, n, 16)
    assert np.array_equal(host(x)[0], xh)
    acc = fk.Accumulator(1, M_SWEEP, 16, 1e-6, "mixed")
    acc.add(x, y, amax)
    theta, rep = acc.fit_sobolev(1.0, LAMBDAS, report=True)
    acc.close()
    assert theta.shape == (256, 16, 2 * M_SWEEP + 1)
    assert rep["n_used"] == n
    th = host(theta)
    xd = xh[None, :].astype(np.float64)
    A0 = O.toeplitz_matrix(O.moments(xd, M_SWEEP), 1, M_SWEEP)
    bo = O.rhs(xd, yh.astype(np.float64), M_SWEEP)
    for li in (0, 85, 170, 255):
        W = O.penalty_sobolev(1, M_SWEEP, LAMBDAS[li], 1.0)
        tho = O.solve_hpd(A0 + np.diag(W), bo.T).T
        for t in range(16):
            assert rel(th[li, t], tho[t]) < 1e-5, (li, t)


def fourier_coeffs_fstar(m):
    """theta*_k of f*(x) = sign(x)|x|^0.7 on [-pi, pi): (1/2pi) int f e^{-ikx} dx
    = -(i/pi) int_0^pi x^0.7 sin(kx) dx (f is odd), by oscillatory quadrature."""
    from scipy.integrate import quad
    th = np.zeros(2 * m + 1, dtype=np.complex128)
    for k in range(1, m + 1):
        val, _ = quad(lambda t: t ** 0.7, 0.0, math.pi, weight="sin", wvar=k, limit=200)
        th[m + k] = -1j * val / math.pi
        th[m - k] = np.conj(th[m + k])
    return th


def test_sweep_full_size_against_closed_form():
    # 1e10 points in 2^28-point chunks, 256 lambdas x 16 targets from one spreading pass.
    # With T ~ I (points fill the period) theta_hat_k = theta*_k / (1 + W_k) up to the
    # sampling error ~ 0.2 / sqrt(n) = 2e-6 per coefficient and the NUFFT error.
    n_total = 10_000_000_000
    chunk = 1 << 28
    acc = fk.Accumulator(1, M_SWEEP, 16, 1e-6, "mixed")
    x = torch.empty((1, chunk), dtype=torch.float32, device="cuda")
    y = torch.empty((16, chunk), dtype=torch.float32, device="cuda")
    amax = torch.empty(16, dtype=torch.int32, device="cuda")
    first = 0
    while first < n_total:
        c = min(chunk, n_total - first)
        xs, ys = x[:, :c], y[:, :c]
        if c != chunk:
            xs = torch.empty((1, c), dtype=torch.float32, device="cuda")
            ys = torch.empty((16, c), dtype=torch.float32, device="cuda")
        fk.generate_sweep_1d(first, c, 16, out=(xs, ys, amax))
        acc.add(xs, ys, amax)
        first += c
    theta = host(acc.fit_sobolev(1.0, LAMBDAS))
    acc.close()
    ths = fourier_coeffs_fstar(M_SWEEP)
    k = np.arange(-M_SWEEP, M_SWEEP + 1, dtype=np.float64)
    worst = 0.0
    for li, lam in enumerate(LAMBDAS):
        want = ths / (1.0 + lam * (1.0 + k ** 2))
        worst = max(worst, float(np.max(np.abs(theta[li] - want[None, :]))))
    assert worst < 3e-5, worst
    # Hermitian symmetry of every fit (real predictions)
    assert np.max(np.abs(theta[:, :, ::-1] - np.conj(theta))) < 1e-12
