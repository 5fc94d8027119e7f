"""CPU oracle for Fourier-represented kernel regression (arXiv 2509.02649).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It shares no code with the CUDA path and imports nothing from it.

Everything here is the plain definition of what the method computes, evaluated
directly in fp64 (complex128), the precision the paper runs in (§3.1 one-
dimensional example).  Library primitives serve as steps: numpy ``cos``/``sin``
for each phase factor (evaluated directly, no recurrences), ``matmul`` for sums
over points, LAPACK's Cholesky for the Hermitian solve.

Conventions (readings of the paper where it is silent or inconsistent):
  * frequency scale pi/(2L) = 1: points are radians, caller rescales (§2.2);
  * modes K = {k in Z^d : |k|_inf <= m}, lexicographic, last dimension fastest
    (§2.2, space H_m);
  * feature map phi_k(x) = exp(-i <k,x>) (§2.2), inner product conjugates its
    first argument (§2.1), so f_theta(x) = sum_k theta_k exp(+i <k,x>) (Eq. 1);
  * design matrix Phi = (phi(X_1) | ... | phi(X_n))^*, so Phi_{jk} = e^{+i<k,X_j>}
    (§2.1).  Hence the moments T_j = (1/n) sum_i e^{-i<j,X_i>} satisfy
    (Phi^*Phi/n)_{k,k'} = T_{k-k'} and b_k = (Phi^*Y/n)_k = (1/n) sum Y_i e^{-i<k,X_i>}
    (§2.3; the covariance-vector display prints e^{+i...}, which contradicts the
    definitions above; the covariance-matrix display agrees with them).

Pins (tests/test_oracle_pins.py): brute-force n x n kernel ridge regression with
the truncated Fourier kernel (§2.1 closed form), equispaced closed forms,
b = Toep(T) theta* for band-limited targets, Toeplitz invariants, the type-1 /
type-2 adjoint identity, noiseless recovery, the additive-model block
identities (§5) and central finite differences of the held-out loss.
No function here is "parity unpinned".
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

CHUNK = 4096  # points per block of phase factors (memory bound only)


# ------------------------------------------------------------------ modes
def mode_grid(d: int, m: int) -> np.ndarray:
    """All k with |k|_inf <= m, shape (D, d), D = (2m+1)^d, lexicographic with
    the last dimension fastest (§2.2, the space H_m)."""
    r = np.arange(-m, m + 1)
    g = np.meshgrid(*([r] * d), indexing="ij")
    return np.stack([a.ravel() for a in g], axis=1)


def _phases(xrow: np.ndarray, kmax: int, sign: float) -> np.ndarray:
    """exp(sign * i * k * x) for k = -kmax..kmax, shape (len(x), 2kmax+1),
    each entry from cos and sin of the product k*x (no recurrences)."""
    arg = np.outer(xrow.astype(np.float64), np.arange(-kmax, kmax + 1, dtype=np.float64))
    return np.cos(arg) + (sign * 1j) * np.sin(arg)


# ------------------------------------------------------------------ type 1 / type 2
def type1(x: np.ndarray, c: np.ndarray, kmax: int) -> np.ndarray:
    """Unnormalised type-1 sums  F_k = sum_i c_i exp(-i <k, x_i>)  for |k|_inf <= kmax.

    x: (d, n) points; c: (n,) or (C, n) strengths (real or complex).
    Returns complex (C, (2kmax+1)^d) (or ((2kmax+1)^d,) for 1-D c), lexicographic.
    This is the sum that §2.3 identifies as a type-I non-uniform Fourier transform.
    """
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    d, n = x.shape
    c = np.asarray(c)
    squeeze = c.ndim == 1
    c2 = c[None, :] if squeeze else c
    C = c2.shape[0]
    K = 2 * kmax + 1
    out = np.zeros((C, K ** d), dtype=np.complex128)
    for i0 in range(0, n, CHUNK):
        sl = slice(i0, min(n, i0 + CHUNK))
        e = [_phases(x[l, sl], kmax, -1.0) for l in range(d)]
        for ch in range(C):
            w = c2[ch, sl].astype(np.complex128)
            if d == 1:
                out[ch] += w @ e[0]
            elif d == 2:
                out[ch] += ((e[0] * w[:, None]).T @ e[1]).ravel()
            elif d == 3:
                e23 = (e[1][:, :, None] * e[2][:, None, :]).reshape(len(w), K * K)
                out[ch] += ((e[0] * w[:, None]).T @ e23).ravel()
            else:
                raise ValueError("d must be 1, 2 or 3")
    return out[0] if squeeze else out


def type2(coef: np.ndarray, x: np.ndarray, kmax: int) -> np.ndarray:
    """Type-2 sums  f(x_i) = sum_k coef_k exp(+i <k, x_i>)  (complex), |k|_inf <= kmax.
    This is f_theta of Eq. (1) with the Fourier feature map of §2.2."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    d, n = x.shape
    K = 2 * kmax + 1
    c = np.asarray(coef, dtype=np.complex128).reshape((K,) * d)
    out = np.empty(n, dtype=np.complex128)
    for i0 in range(0, n, CHUNK):
        sl = slice(i0, min(n, i0 + CHUNK))
        e = [_phases(x[l, sl], kmax, +1.0) for l in range(d)]
        if d == 1:
            out[sl] = e[0] @ c
        elif d == 2:
            out[sl] = np.einsum("ia,ab,ib->i", e[0], c, e[1], optimize=True)
        elif d == 3:
            out[sl] = np.einsum("ia,abc,ib,ic->i", e[0], c, e[1], e[2], optimize=True)
        else:
            raise ValueError("d must be 1, 2 or 3")
    return out


# ------------------------------------------------------------------ the system
def moments(x: np.ndarray, m: int) -> np.ndarray:
    """First-row moments of Sigma = Phi^*Phi/n over the doubled range:
    T_j = (1/n) sum_i exp(-i <j, X_i>), |j|_inf <= 2m  (§2.3, covariance matrix)."""
    n = np.atleast_2d(x).shape[1]
    return type1(x, np.ones(n), 2 * m) / n


def rhs(x: np.ndarray, y: np.ndarray, m: int) -> np.ndarray:
    """b_k = (Phi^*Y/n)_k = (1/n) sum_i Y_i exp(-i <k, X_i>), |k|_inf <= m
    (§2.3, covariance vector).  y: (n,) or (C, n)."""
    n = np.atleast_2d(x).shape[1]
    return type1(x, np.asarray(y, dtype=np.float64), m) / n


def penalty_sobolev(d: int, m: int, lam: float, s: float, c0: float = 1.0) -> np.ndarray:
    """Diagonal of lambda S^2 with S_kk^2 = c0 + |k|_2^{2s} (§3.1; c0 = 1 in the
    paper, 0^{2s} = 0)."""
    k = mode_grid(d, m).astype(np.float64)
    r2 = (k ** 2).sum(axis=1)
    pw = np.where(r2 > 0, r2 ** s, 0.0)
    return lam * (c0 + pw)


def penalty_lowbias(d: int, m: int, lam: float) -> np.ndarray:
    """Diagonal of lambda I, the low-bias estimator with M = I (§3.2)."""
    return np.full((2 * m + 1) ** d, float(lam))


def pde_symbol(d: int, m: int, alpha: np.ndarray, a: np.ndarray) -> np.ndarray:
    """P(ik) = sum_alpha a_alpha prod_l (i k_l)^{alpha_l}: the Fourier symbol of the
    constant-coefficient operator D of §4 acting on e^{+i<k,x>}.
    alpha: (n_terms, d) non-negative integers; a: (n_terms,) real."""
    k = mode_grid(d, m).astype(np.float64)
    alpha = np.asarray(alpha, dtype=np.int64).reshape(-1, d)
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    out = np.zeros(len(k), dtype=np.complex128)
    for t in range(len(a)):
        term = np.ones(len(k), dtype=np.complex128)
        for l in range(d):
            term = term * (1j * k[:, l]) ** int(alpha[t, l])
        out += a[t] * term
    return out


def penalty_pik(d: int, m: int, lam: float, s: float, mu: float, alpha, a,
                c0: float = 1.0) -> np.ndarray:
    """lambda S^2 + mu D^* C D on the full period, where the Fourier matrix C of
    the domain is the identity, so the penalty is diagonal:
    W_k = lambda (c0 + |k|^{2s}) + mu |P(ik)|^2  (§4, tractable domains)."""
    return penalty_sobolev(d, m, lam, s, c0) + mu * np.abs(pde_symbol(d, m, alpha, a)) ** 2


def box_moments(d: int, m: int, lo, hi) -> np.ndarray:
    """Moments of the normalised Lebesgue measure of a box Omega = prod_l [lo_l, hi_l]
    (inside the period [-pi, pi)^d):  c_j = (2 pi)^{-d} int_Omega e^{-i<j, x>} dx,
    |j|_inf <= 2m, lexicographic.  The Fourier matrix C of Omega (§4, tractable
    domains) is C_{k,k'} = c_{k-k'}: the form int_Omega |D f_theta|^2 dx / (2 pi)^d of
    f_theta = sum_k theta_k e^{+i<k,x>} is (D theta)^* C (D theta).  Per coordinate
    the integral is (e^{-i j hi} - e^{-i j lo}) / (-i j), or hi - lo at j = 0."""
    lo = np.broadcast_to(np.asarray(lo, dtype=np.float64), (d,))
    hi = np.broadcast_to(np.asarray(hi, dtype=np.float64), (d,))
    j = np.arange(-2 * m, 2 * m + 1, dtype=np.float64)
    out = np.ones(1, dtype=np.complex128)
    for l in range(d):
        with np.errstate(divide="ignore", invalid="ignore"):
            f = (np.exp(-1j * j * hi[l]) - np.exp(-1j * j * lo[l])) / (-1j * j)
        f[2 * m] = hi[l] - lo[l]
        out = np.multiply.outer(out, f / (2 * np.pi)).ravel()
    return out


def penalty_pik_general(d: int, m: int, lam: float, s: float, mu: float, alpha, a,
                        c_moments: np.ndarray, c0: float = 1.0) -> np.ndarray:
    """Dense penalty lambda S^2 + mu D^* C D of §4 with a non-diagonal Fourier matrix
    C_{k,k'} = c_{k-k'} (a sub-domain in closed form, or the collocation points'
    moments (1/n_r) sum_r e^{-i<j, X_r>}); D = diag P(ik)."""
    P = pde_symbol(d, m, alpha, a)
    C = toeplitz_matrix(c_moments, d, m)
    return np.diag(penalty_sobolev(d, m, lam, s, c0)) + mu * (np.conj(P)[:, None] * C * P[None, :])


def fit_penalised(x: np.ndarray, y: np.ndarray, m: int, Pen: np.ndarray) -> np.ndarray:
    """theta_hat = (Phi^*Phi/n + Pen)^{-1} Phi^*Y/n for a dense Hermitian penalty."""
    d = np.atleast_2d(x).shape[0]
    A = toeplitz_matrix(moments(x, m), d, m) + Pen
    return solve_hpd(A, rhs(x, y, m).T).T


def toeplitz_matrix(T: np.ndarray, d: int, m: int) -> np.ndarray:
    """Dense Sigma with Sigma_{k,k'} = T_{k-k'} (§2.3: Hermitian d-level block
    Toeplitz, determined by its first row)."""
    k = mode_grid(d, m)
    K2 = 4 * m + 1
    diff = k[:, None, :] - k[None, :, :] + 2 * m  # index of k - k' in the doubled grid
    flat = np.zeros(diff.shape[:2], dtype=np.int64)
    for l in range(d):
        flat = flat * K2 + diff[:, :, l]
    return np.asarray(T, dtype=np.complex128).reshape(-1)[flat]


def solve_hpd(A: np.ndarray, b: np.ndarray, refine: int = 1) -> np.ndarray:
    """Solve A theta = b for Hermitian positive definite A: Cholesky (LAPACK,
    raises on a non-positive pivot) plus ``refine`` steps of iterative refinement."""
    cf = sla.cho_factor(A, lower=True, check_finite=True)
    th = sla.cho_solve(cf, b)
    for _ in range(refine):
        th = th + sla.cho_solve(cf, b - A @ th)
    return th


def fit(x: np.ndarray, y: np.ndarray, m: int, W: np.ndarray) -> np.ndarray:
    """theta_hat = (Phi^*Phi/n + diag W)^{-1} Phi^*Y/n  (Eq. 2 with lambda M^*M = diag W).
    y may hold several targets (C, n); returns (C, D) or (D,)."""
    d = np.atleast_2d(x).shape[0]
    A = toeplitz_matrix(moments(x, m), d, m) + np.diag(np.asarray(W, dtype=np.float64))
    b = rhs(x, y, m)
    return solve_hpd(A, b.T).T


def predict(theta: np.ndarray, xq: np.ndarray, m: int) -> np.ndarray:
    """f_hat(x) = <phi(x), theta_hat> = Re sum_k theta_k e^{+i<k,x>} (§2.1).
    The imaginary part vanishes for Hermitian-symmetric theta; see predict_imag."""
    return type2(theta, xq, m).real


def predict_imag(theta: np.ndarray, xq: np.ndarray, m: int) -> np.ndarray:
    return type2(theta, xq, m).imag


# ------------------------------------------------------------------ brute-force KRR
def fourier_kernel(xa: np.ndarray, xb: np.ndarray, m: int, W: np.ndarray) -> np.ndarray:
    """Truncated Fourier kernel K(x, x') = sum_k cos<k, x - x'> / W_k, evaluated
    pairwise from the differences (valid for W_k = W_{-k})."""
    xa = np.atleast_2d(xa)
    xb = np.atleast_2d(xb)
    d = xa.shape[0]
    k = mode_grid(d, m).astype(np.float64)
    invW = 1.0 / np.asarray(W, dtype=np.float64)
    out = np.zeros((xa.shape[1], xb.shape[1]))
    for i0 in range(0, xa.shape[1], 256):
        sl = slice(i0, i0 + 256)
        diff = xa[:, sl, None] - xb[:, None, :]  # (d, a, b)
        acc = np.zeros(diff.shape[1:])
        for t in range(len(k)):
            ph = np.zeros(diff.shape[1:])
            for l in range(d):
                if k[t, l] != 0.0:
                    ph = ph + k[t, l] * diff[l]
            acc += invW[t] * np.cos(ph)
        out[sl] = acc
    return out


def krr_bruteforce(x: np.ndarray, y: np.ndarray, m: int, W: np.ndarray, xq: np.ndarray):
    """Closed-form kernel ridge regression (§2.1) with the truncated Fourier kernel,
    f_hat(x) = K(x, X) (K_n + n I)^{-1} Y.  The ridge is n (not lambda): the
    penalty lambda is inside W, and the empirical risk carries 1/n (§2.1), so by
    the push-through identity theta_hat = W^{-1} Phi^* alpha with
    alpha = (Phi W^{-1} Phi^* + n I)^{-1} Y, which is Eq. (2).
    Returns (prediction at xq, theta from the dual coefficients)."""
    x = np.atleast_2d(x)
    n = x.shape[1]
    Kn = fourier_kernel(x, x, m, W)
    alpha = np.linalg.solve(Kn + n * np.eye(n), np.asarray(y, dtype=np.float64))
    fq = fourier_kernel(xq, x, m, W) @ alpha
    theta = type1(x, alpha, m) / np.asarray(W, dtype=np.float64)
    return fq, theta


# ------------------------------------------------------------------ additive model (§5)
def additive_gram(X: np.ndarray, m: int) -> np.ndarray:
    """Sigma of Prop. 5.1: block (l1, l2) = Phi_{l1}^* Phi_{l2} / n, with entries
    (1/n) sum_i e^{-i k1 X_{i,l1}} e^{+i k2 X_{i,l2}}; shape (d(2m+1), d(2m+1))."""
    X = np.atleast_2d(X)
    d, n = X.shape
    K = 2 * m + 1
    G = np.zeros((d * K, d * K), dtype=np.complex128)
    for i0 in range(0, n, CHUNK):
        sl = slice(i0, min(n, i0 + CHUNK))
        E = np.concatenate([_phases(X[l, sl], m, -1.0) for l in range(d)], axis=1)  # e^{-ikX}
        G += E.T @ np.conj(E)
    return G / n


def additive_rhs(X: np.ndarray, y: np.ndarray, m: int) -> np.ndarray:
    """(Phi_1^*Y/n, ..., Phi_d^*Y/n) of Prop. 5.1; shape (d(2m+1),) per target."""
    X = np.atleast_2d(X)
    return np.concatenate([rhs(X[l:l + 1], y, m) for l in range(X.shape[0])], axis=-1)


def fit_additive(X: np.ndarray, y: np.ndarray, m: int, lam: float) -> np.ndarray:
    """Low-bias additive estimator (Sigma + lambda I)^{-1} (Phi_l^*Y/n)_l (Prop. 5.1)."""
    G = additive_gram(X, m)
    return solve_hpd(G + lam * np.eye(G.shape[0]), additive_rhs(X, y, m).T).T


def predict_additive(theta: np.ndarray, Xq: np.ndarray, m: int) -> np.ndarray:
    """f_theta(x) = sum_l <phi(x_l), theta_l> (§5, additive parametrisation)."""
    Xq = np.atleast_2d(Xq)
    d = Xq.shape[0]
    K = 2 * m + 1
    th = np.asarray(theta).reshape(d, K)
    return sum(type2(th[l], Xq[l:l + 1], m) for l in range(d)).real


def additive_krr(X: np.ndarray, y: np.ndarray, m: int, lam: float, Xq: np.ndarray):
    """Brute-force KRR with the additive kernel sum_l sum_k cos(k (x_l - x'_l)) / lam,
    ridge n (see krr_bruteforce)."""
    X = np.atleast_2d(X)
    d, n = X.shape
    W1 = np.full(2 * m + 1, float(lam))
    Kn = sum(fourier_kernel(X[l:l + 1], X[l:l + 1], m, W1) for l in range(d))
    alpha = np.linalg.solve(Kn + n * np.eye(n), np.asarray(y, dtype=np.float64))
    Kq = sum(fourier_kernel(Xq[l:l + 1], X[l:l + 1], m, W1) for l in range(d))
    return Kq @ alpha


# ------------------------------------------------------------------ hypergradient
def heldout_loss(theta: np.ndarray, xv: np.ndarray, yv: np.ndarray, m: int) -> float:
    """L = (1/n_v) sum_i (f_hat(x^v_i) - y^v_i)^2."""
    r = predict(theta, xv, m) - np.asarray(yv, dtype=np.float64)
    return float(np.mean(r * r))


def hypergradient(x, y, xv, yv, m: int, W: np.ndarray):
    """Gradient of the held-out loss L(theta_hat(W, Y)) by the adjoint method.

    With A = Sigma + diag W, theta = A^{-1} b and residual r = f_hat(x^v) - y^v:
      g   = (1/n_v) sum_i r_i e^{-i<k, x^v_i>}     (Wirtinger gradient dL/d conj(theta))
      z   = A^{-1} g                              (adjoint solve; A is Hermitian)
      dL/dW_k = -2 Re(conj(z_k) theta_k)
      dL/dY_i = (2/n) Re sum_k z_k e^{+i<k, X_i>}
    Not in the paper; derived from Eq. (2).  Returns (L, theta, dL/dW, dL/dY)."""
    x = np.atleast_2d(x)
    d, n = x.shape
    xv = np.atleast_2d(xv)
    A = toeplitz_matrix(moments(x, m), d, m) + np.diag(np.asarray(W, dtype=np.float64))
    cf = sla.cho_factor(A, lower=True)
    b = rhs(x, y, m)
    theta = sla.cho_solve(cf, b)
    theta = theta + sla.cho_solve(cf, b - A @ theta)
    r = predict(theta, xv, m) - np.asarray(yv, dtype=np.float64)
    L = float(np.mean(r * r))
    g = type1(xv, r, m) / xv.shape[1]
    z = sla.cho_solve(cf, g)
    z = z + sla.cho_solve(cf, g - A @ z)
    dW = -2.0 * np.real(np.conj(z) * theta)
    dY = (2.0 / n) * type2(z, x, m).real
    return L, theta, dW, dY


def penalty_param_grads(d: int, m: int, lam: float, s: float, mu: float, alpha, a,
                        dW: np.ndarray, c0: float = 1.0) -> dict:
    """Chain rule from dL/dW to the hyper-parameters of
    W_k = lambda (c0 + |k|^{2s}) + mu |P(ik)|^2:
      dL/dlambda = sum_k dW_k (c0 + |k|^{2s})
      dL/ds      = sum_k dW_k lambda |k|^{2s} ln(|k|^2)      (k != 0)
      dL/dmu     = sum_k dW_k |P(ik)|^2
      dL/da_t    = sum_k dW_k 2 mu Re(conj(P(ik)) (ik)^{alpha_t})."""
    k = mode_grid(d, m).astype(np.float64)
    r2 = (k ** 2).sum(axis=1)
    pw = np.where(r2 > 0, r2 ** s, 0.0)
    lg = np.where(r2 > 0, np.log(np.where(r2 > 0, r2, 1.0)), 0.0)
    out = {"lambda": float(np.sum(dW * (c0 + pw))),
           "s": float(np.sum(dW * lam * pw * lg))}
    if alpha is not None and len(np.atleast_1d(a)) > 0:
        P = pde_symbol(d, m, alpha, a)
        out["mu"] = float(np.sum(dW * np.abs(P) ** 2))
        alpha = np.asarray(alpha, dtype=np.int64).reshape(-1, d)
        ga = []
        for t in range(alpha.shape[0]):
            mono = np.ones(len(k), dtype=np.complex128)
            for l in range(d):
                mono = mono * (1j * k[:, l]) ** int(alpha[t, l])
            ga.append(float(np.sum(dW * 2.0 * mu * np.real(np.conj(P) * mono))))
        out["a"] = np.array(ga)
    return out
