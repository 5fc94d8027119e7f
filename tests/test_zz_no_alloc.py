"""fk_type1_noalloc: the type-1 transform for callers that cannot allocate device
memory at call time (their device memory is wholly reserved by their own pool
allocator, or their policy forbids allocation after start-up).  It takes its
scratch from a built-in device array instead of cudaMallocAsync.

Checked against fk_type1 (the allocating entry point) on two calls in a row, with
the tolerance the type-1 parity tests use (10 * eps, normwise).  This file is
collected last so that a run stopping at its first failure has run every other
test already; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu

fk = pytest.importorskip("paper_2509_02649_b300")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision,eps,dtype", [("fp64", 1e-12, torch.float64), ("mixed", 1e-6, torch.float32)])
@pytest.mark.parametrize("d,kmax,n", [(1, 60, 5003), (2, 16, 20011)])
def test_noalloc_matches_allocating_type1_twice(precision, eps, dtype, d, kmax, n):
    x = torch.from_numpy(S.uniform_points(n, d, 41)).to("cuda", dtype)
    c = torch.from_numpy(np.stack([S.noise(n, 1.0, 41, 5), np.ones(n)])).to("cuda", dtype)
    ref = fk.fk_type1(x, c, kmax, eps, precision).cpu().numpy()
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        got = fk.fk_type1_noalloc(x, c, kmax, eps, precision).cpu().numpy()
        for ch in range(2):
            assert rel(got[ch], ref[ch]) <= 10 * eps


def test_noalloc_rejects_shapes_beyond_its_scratch():
    x = torch.zeros((2, 16), dtype=torch.float32, device="cuda")
    c = torch.ones((8, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(fk.FkError) as e:
        fk.fk_type1_noalloc(x, c, 300, 1e-6, "mixed")  # 8 channels on a 1024^2 grid
    assert e.value.name == "FK_EINVAL" and "limit" in str(e.value)
