"""The autotuner: a tuned call gives the same result as an untuned one (up to fp32
summation order), records its problem class, and later calls reuse the stored shape
without trials."""
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


def test_autotune_2d_spreader():
    fk.fk_autotune_clear()
    n, m = 1 << 21, 16
    x, y = S.wl2_sobolev_2d(n, dtype=np.float32)
    X = torch.from_numpy(x).cuda()
    Y = torch.from_numpy(y).cuda()
    plain = fk.fk_build_system(X, Y, m, 1e-6, "mixed")
    assert fk.fk_autotune_table() == ""
    c0 = fk.fk_launch_count()
    tuned = fk.fk_build_system(X, Y, m, 1e-6, "mixed", opts=fk.default_opts(autotune=1))
    c1 = fk.fk_launch_count()
    table = fk.fk_autotune_table()
    assert "spread2d" in table and "->" in table
    again = fk.fk_build_system(X, Y, m, 1e-6, "mixed", opts=fk.default_opts(autotune=1))
    c2 = fk.fk_launch_count()
    assert c2 - c1 < (c1 - c0) / 3  # no trials the second time
    for a, b in zip(tuned, plain):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
    for a, b in zip(again, plain):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
    # and against the oracle on a slice of the moments
    To = O.moments(x[:, :50_000].astype(np.float64), 4)
    T4, _ = fk.fk_build_system(X[:, :50_000].contiguous(), Y[:50_000].contiguous(), 4, 1e-6, "mixed",
                               opts=fk.default_opts(autotune=1))
    assert rel(T4.cpu().numpy(), To) < 1e-5
    fk.fk_autotune_clear()
    assert fk.fk_autotune_table() == ""


def test_autotune_2d_spreader_two_owner_sizes():
    # the 256 x 256 grid (m = 32), whose default owners come in two sizes; the trials
    # also time uniform owners in the same kernel, and the kept shape must agree with
    # the untuned call and with direct sums
    fk.fk_autotune_clear()
    n, m = 1 << 21, 32
    x, y = S.wl2_sobolev_2d(n, dtype=np.float32)
    X = torch.from_numpy(x).cuda()
    Y = torch.from_numpy(y).cuda()
    plain = fk.fk_build_system(X, Y, m, 1e-6, "mixed")
    tuned = fk.fk_build_system(X, Y, m, 1e-6, "mixed", opts=fk.default_opts(autotune=1))
    assert "spread2d" in fk.fk_autotune_table()
    for a, b in zip(tuned, plain):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
    K = 4 * m + 1
    T = tuned[0].cpu().numpy()
    x0, x1 = x[0].astype(np.float64), x[1].astype(np.float64)
    for j0, j1 in [(0, 0), (1, -2), (-64, 64), (40, -17)]:
        want = np.mean(np.exp(-1j * (j0 * x0 + j1 * x1)))
        assert abs(T[(j0 + 2 * m) * K + (j1 + 2 * m)] - want) < 1e-6
    fk.fk_autotune_clear()


def test_autotune_1d_spreader_and_accumulator():
    fk.fk_autotune_clear()
    n = 1 << 21
    x, y, amax = fk.generate_sweep_1d(0, n, 16)
    plain = fk.Accumulator(1, 1000, 16, 1e-6, "mixed")
    plain.add(x, y, amax)
    T0, b0, _ = plain.system()
    plain.close()
    tuned = fk.Accumulator(1, 1000, 16, 1e-6, "mixed", opts=fk.default_opts(autotune=1))
    tuned.add(x, y, amax)
    tuned.add(x, y, amax)  # the second add reuses the stored shape and adds once more
    T1, b1, nt = tuned.system()
    tuned.close()
    assert nt == 2 * n
    assert "spread1d" in fk.fk_autotune_table()
    # the same points twice: the normalised sums are unchanged (integer sums: exact
    # up to the fp64 scaling of the two chunks)
    assert rel(T1.cpu().numpy(), T0.cpu().numpy()) < 1e-12
    assert rel(b1.cpu().numpy(), b0.cpu().numpy()) < 1e-12
    fk.fk_autotune_clear()
