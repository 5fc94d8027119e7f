"""Host twin of the counter-based sweep generator (CPU).

Philox4x32-10 is pinned to the published known-answer vectors of its authors'
reference distribution (Random123); the sample it drives is checked for chunk
independence and for the distribution the 1-D sweep workload states.
"""
import numpy as np
import pytest

import synthetic as S

# Philox4x32-10 known-answer vectors: (counter, key) -> output
KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF), (0xFFFFFFFF, 0xFFFFFFFF),
     (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,want", KAT)
def test_philox_known_answers(ctr, key, want):
    out = S.philox4x32_10(np.array(ctr, dtype=np.uint32).reshape(4, 1), key)[:, 0]
    assert [int(v) for v in out] == list(want)


def test_philox_vectorised_matches_single():
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(4, 50), dtype=np.uint64).astype(np.uint32)
    many = S.philox4x32_10(ctr, (123, 456))
    for c in range(50):
        one = S.philox4x32_10(ctr[:, c:c + 1], (123, 456))[:, 0]
        assert np.array_equal(one, many[:, c])


def test_sweep_chunks_are_independent():
    # any split of the index range reproduces the same sample
    x, y = S.sweep_counter_points(0, 4000, 3)
    for cut in (4, 1000, 1337, 2400):
        xa, ya = S.sweep_counter_points(0, cut, 3)
        xb, yb = S.sweep_counter_points(cut, 4000 - cut, 3)
        assert np.array_equal(np.concatenate([xa, xb]), x)
        assert np.array_equal(np.concatenate([ya, yb], axis=1), y)


def test_sweep_distribution():
    n = 200_000
    x, y = S.sweep_counter_points(1 << 28, n, 4)
    assert x.dtype == np.float32 and y.dtype == np.float32
    assert np.all(x > -np.float32(np.pi)) and np.all(x < np.float32(np.pi))
    # uniform on (-pi, pi): mean 0, variance pi^2 / 3
    assert abs(x.mean()) < 5 * np.pi / np.sqrt(3 * n)
    assert abs(x.var() / (np.pi ** 2 / 3) - 1) < 0.02
    xd = x.astype(np.float64)
    fstar = np.sign(xd) * np.abs(xd) ** 0.7
    z = (y.astype(np.float64) - fstar) / 0.2
    for t in range(4):
        assert abs(z[t].mean()) < 5 / np.sqrt(n)
        assert abs(z[t].var() - 1) < 0.02
        # fourth moment of a standard normal is 3
        assert abs((z[t] ** 4).mean() - 3) < 0.1
    # the targets' noise streams are independent
    c = np.corrcoef(z)
    assert np.max(np.abs(c - np.eye(4))) < 5 / np.sqrt(n)


def test_sweep_uniform_is_exact_in_fp32():
    # X = fp32(u 2pi_f - pi_f) is a single rounding of the exact value
    x, _ = S.sweep_counter_points(0, 64, 0)
    w = S.philox4x32_10(np.array([[0] * 16, [0] * 16, [0] * 16, [0] * 16], dtype=np.uint32)
                        + np.array([np.arange(16), [0] * 16, [0] * 16, [0] * 16], dtype=np.uint32), (S.SEED, 5))
    words = w.T.reshape(-1)  # point 4j + r takes word r of counter j
    u = ((words >> 9).astype(np.float64) + 0.5) * 2.0 ** -23
    assert np.all(u.astype(np.float32).astype(np.float64) == u)
    exact = u * np.float64(np.float32(2 * np.pi)) - np.float64(np.float32(np.pi))
    assert np.array_equal(x, exact.astype(np.float32))
