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
