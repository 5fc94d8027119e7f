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
