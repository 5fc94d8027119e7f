"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and evaluates the target functions that
define each workload; it holds none of the estimator's arithmetic.  Both the
CPU oracle (``oracle/``) and the CUDA path's tests and benchmark take their
inputs from here.

Streams are numpy ``Philox`` generators keyed by ``(seed, workload, stream)``:
stream 0 draws the points X, stream ``1 + t`` the noise of target ``t`` and
stream 100 the held-out validation set.

Points are returned structure-of-arrays, shape ``(d, n)``, in radians on
``[-pi, pi)`` (frequency scale ``pi / (2L) = 1``).
"""
from __future__ import annotations

import numpy as np

SEED = 20250902
TWO_PI = 2.0 * np.pi


def generator(workload: int, stream: int, seed: int = SEED) -> np.random.Generator:
    key = np.array([seed, (workload << 32) | stream], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def uniform_points(n: int, d: int, workload: int, stream: int = 0,
                   dtype=np.float64, seed: int = SEED) -> np.ndarray:
    """X ~ Uniform[-pi, pi)^d, SoA (d, n)."""
    g = generator(workload, stream, seed)
    x = g.random((d, n), dtype=np.float64) * TWO_PI - np.pi
    return x.astype(dtype, copy=False)


def noise(n: int, sigma: float, workload: int, stream: int, seed: int = SEED) -> np.ndarray:
    g = generator(workload, stream, seed)
    return sigma * g.standard_normal(n)


# ---------------------------------------------------------------- workloads
# 1: 1-D Sobolev, plain FP64:  Y = sin(3X) + 0.5 cos(7X) + N(0, 0.1^2)
def wl1_sobolev_1d(n: int, dtype=np.float64, seed: int = SEED):
    x = uniform_points(n, 1, 1, 0, np.float64, seed)
    y = np.sin(3 * x[0]) + 0.5 * np.cos(7 * x[0]) + noise(n, 0.1, 1, 1, seed)
    return x.astype(dtype), y.astype(dtype)


# 2: 2-D Sobolev:  Y = exp(-|X|^2) + N(0, 0.05^2)
def wl2_sobolev_2d(n: int, dtype=np.float32, seed: int = SEED):
    x = uniform_points(n, 2, 2, 0, np.float64, seed)
    y = np.exp(-(x[0] ** 2 + x[1] ** 2)) + noise(n, 0.05, 2, 1, seed)
    return x.astype(dtype), y.astype(dtype)


# 3: 2-D physics-informed (t, x), heat prior:  Y = exp(-0.1 t) sin(x) + N(0, 0.1^2)
def wl3_pik_heat(n: int, dtype=np.float32, seed: int = SEED, validation: bool = False):
    stream = 100 if validation else 0
    x = uniform_points(n, 2, 3, stream, np.float64, seed)
    y = np.exp(-0.1 * x[0]) * np.sin(x[1]) + noise(n, 0.1, 3, stream + 1, seed)
    return x.astype(dtype), y.astype(dtype)


# 4: additive d=8:  Y = sum_j sin((j+1) X_j) / (j+1) + N(0, 0.1^2)
def wl4_additive(n: int, d: int = 8, dtype=np.float32, seed: int = SEED):
    x = uniform_points(n, d, 4, 0, np.float64, seed)
    y = sum(np.sin((j + 1) * x[j]) / (j + 1) for j in range(d)) + noise(n, 0.1, 4, 1, seed)
    return x.astype(dtype), y.astype(dtype)


# 5: 1-D at scale, 16 targets:  Y_t = sign(X)|X|^0.7 + N(0, 0.2^2), t = 0..15
def wl5_sweep_1d(n: int, n_targets: int = 16, dtype=np.float32, seed: int = SEED):
    x = uniform_points(n, 1, 5, 0, np.float64, seed)
    f = np.sign(x[0]) * np.abs(x[0]) ** 0.7
    y = np.stack([f + noise(n, 0.2, 5, 1 + t, seed) for t in range(n_targets)])
    return x.astype(dtype), y.astype(dtype)


def equispaced_1d(n: int) -> np.ndarray:
    """X_i = -pi + 2 pi i / n, shape (1, n)."""
    return (-np.pi + TWO_PI * np.arange(n) / n)[None, :]


def equispaced_2d(n1: int, n2: int) -> np.ndarray:
    """Tensor grid of equispaced points, shape (2, n1*n2)."""
    a = -np.pi + TWO_PI * np.arange(n1) / n1
    b = -np.pi + TWO_PI * np.arange(n2) / n2
    A, B = np.meshgrid(a, b, indexing="ij")
    return np.stack([A.ravel(), B.ravel()])


def bandlimited_1d(x: np.ndarray) -> np.ndarray:
    """Noiseless band-limited target sin(3x) + 0.5 cos(7x) at x (1, n)."""
    return np.sin(3 * x[0]) + 0.5 * np.cos(7 * x[0])


def bandlimited_2d(x: np.ndarray) -> np.ndarray:
    """Noiseless band-limited target 0.2 + cos(2 x1 + 3 x2) + 0.3 sin(x1 - 5 x2)
    at x (2, n)."""
    return 0.2 + np.cos(2 * x[0] + 3 * x[1]) + 0.3 * np.sin(x[0] - 5 * x[1])


# ---------------------------------------------------------------- counter-based twin
# The 1-D sweep at scale (workload 5, up to 1e10 points) is generated on the device
# in chunks; this is the host twin of that generator, written from the published
# definition of Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random
# numbers: as easy as 1, 2, 3", SC 2011): two 32x32->64 multiplications per round
# with multipliers 0xD2511F53 and 0xCD9E8D57, key schedule bumped by the Weyl
# constants 0x9E3779B9 and 0xBB67AE85, ten rounds.
#
# Draws for point i (j = i // 4, r = i % 4), key (seed mod 2^32, workload):
#   X_i:        word r of Philox(counter = (j mod 2^32, j div 2^32, 0, 0));
#               u = (floor(word / 2^9) + 1/2) 2^-23 (exact in fp32) and
#               X = fp32(u fp32(2 pi) - fp32(pi)) with one rounding.
#   noise z_ti: words (2p, 2p + 1), p = r // 2, of Philox(counter = (.., .., 1 + t, 0))
#               -> uniforms u1, u2 as above; Box-Muller radius sqrt(-2 ln u1) times
#               cos(2 pi u2) for even r, sin(2 pi u2) for odd r.
#   Y_ti = sign(X_i) |X_i|^0.7 + 0.2 z_ti.
# The device computes the transcendental steps in fp32 with CUDA's libm, this twin
# in fp64 rounded to fp32: X agrees bit for bit, Y to a few fp32 ulps.

PHILOX_M = (0xD2511F53, 0xCD9E8D57)
PHILOX_W = (0x9E3779B9, 0xBB67AE85)
TWO_PI_F32 = np.float32(2.0 * np.pi)
PI_F32 = np.float32(np.pi)


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox4x32-10 of counters ctr (4, m) uint32 under key (k0, k1); returns (4, m)."""
    c = [np.asarray(ctr[i], dtype=np.uint64) for i in range(4)]
    k0, k1 = np.uint64(key[0] & 0xFFFFFFFF), np.uint64(key[1] & 0xFFFFFFFF)
    mask = np.uint64(0xFFFFFFFF)
    m0, m1 = np.uint64(PHILOX_M[0]), np.uint64(PHILOX_M[1])
    for rnd in range(10):
        if rnd:
            k0 = (k0 + np.uint64(PHILOX_W[0])) & mask
            k1 = (k1 + np.uint64(PHILOX_W[1])) & mask
        p0 = c[0] * m0
        p1 = c[2] * m1
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ k0) & mask, p1 & mask,
             ((p0 >> np.uint64(32)) ^ c[3] ^ k1) & mask, p0 & mask]
    return np.stack(c).astype(np.uint32)


def _unit_f32(words: np.ndarray) -> np.ndarray:
    """(floor(w / 2^9) + 1/2) 2^-23 in (0, 1), exact in fp32."""
    return ((words >> np.uint32(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def sweep_counter_points(first: int, n: int, n_targets: int = 16, seed: int = SEED,
                         workload: int = 5):
    """Points first .. first + n - 1 of the counter-based 1-D sweep workload.

    Returns X (n,) float32 and Y (n_targets, n) float32."""
    i = np.arange(first, first + n, dtype=np.uint64)
    j = i >> np.uint64(2)
    r = (i & np.uint64(3)).astype(np.int64)
    jlo = (j & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    jhi = (j >> np.uint64(32)).astype(np.uint32)
    key = (seed & 0xFFFFFFFF, workload)
    zeros = np.zeros_like(jlo)
    cols = np.arange(n)
    w = philox4x32_10(np.stack([jlo, jhi, zeros, zeros]), key)
    u = _unit_f32(w[r, cols])
    x = (u * np.float64(TWO_PI_F32) - np.float64(PI_F32)).astype(np.float32)
    xd = x.astype(np.float64)
    fstar = (np.sign(xd) * np.abs(xd) ** 0.7).astype(np.float32)
    y = np.empty((n_targets, n), dtype=np.float32)
    pair = 2 * (r >> 1)
    for t in range(n_targets):
        wt = philox4x32_10(np.stack([jlo, jhi, np.full_like(jlo, 1 + t), zeros]), key)
        u1 = _unit_f32(wt[pair, cols])
        u2 = _unit_f32(wt[pair + 1, cols])
        rad = np.sqrt(-2.0 * np.log(u1)).astype(np.float32).astype(np.float64)
        ang = 2.0 * np.pi * u2
        trig = np.where(r % 2 == 0, np.cos(ang), np.sin(ang)).astype(np.float32).astype(np.float64)
        z = (rad * trig).astype(np.float32).astype(np.float64)
        y[t] = (np.float64(np.float32(0.2)) * z + fstar.astype(np.float64)).astype(np.float32)
    return x, y
