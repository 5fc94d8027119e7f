"""Streaming sums from host memory (fk_accum_add_host): the chunked copies through the
accumulator's staging buffers must give the sums of Sec. 2.3 over all points, as the
oracle computes them, whatever the chunking, the host memory kind (page-locked or
pageable) and the number of calls.

Tolerances: mixed path 1e-5 normwise (as the device-resident accumulator tests),
FP64 path at eps = 1e-12 1e-10 normwise.
"""
import ctypes

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


def host(t):
    return t.detach().cpu().numpy()


def sample(d, n, dtype=np.float32):
    if d == 1:
        x, y = S.sweep_counter_points(0, n, 2)
        return x[None, :].astype(dtype), y.astype(dtype)
    x, y1 = S.wl2_sobolev_2d(n, dtype=dtype)
    return x, y1[None, :]


@pytest.mark.parametrize("d,m,chunk,pinned", [(1, 60, 0, True), (1, 60, 1777, False), (2, 12, 2500, True),
                                              (2, 12, 10 ** 6, False)])
def test_host_chunks_match_oracle(d, m, chunk, pinned):
    n = 10007  # ragged against every chunk size above
    x, y = sample(d, n)
    xh = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    yh = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32))
    if pinned:
        xh, yh = xh.pin_memory(), yh.pin_memory()
    acc = fk.Accumulator(d, m, y.shape[0], 1e-6, "mixed")
    acc.add_host(xh, yh, chunk=chunk)
    T, bb, ntot = acc.system()
    acc.close()
    assert ntot == n
    To = O.moments(x.astype(np.float64), m)
    bo = O.rhs(x.astype(np.float64), y.astype(np.float64), m)
    assert rel(host(T), To) < 1e-5
    assert rel(host(bb), bo) < 1e-5


def test_host_fp64_several_calls_and_growing_chunks():
    # three calls whose chunk grows (the staging buffers are reallocated in between),
    # then a reset and the whole sample again: both equal the oracle's sums
    n, m = 9001, 10
    x, y = sample(2, n, np.float64)
    acc = fk.Accumulator(2, m, 1, 1e-12, "fp64")
    parts = [(0, 2000, 700), (2000, 6000, 1500), (6000, n, 0)]
    for a, b, c in parts:
        acc.add_host(torch.from_numpy(np.ascontiguousarray(x[:, a:b])),
                     torch.from_numpy(np.ascontiguousarray(y[:, a:b])), chunk=c)
    T, bb, ntot = acc.system()
    To = O.moments(x, m)
    bo = O.rhs(x, y, m)
    assert ntot == n
    assert rel(host(T), To) < 1e-10
    assert rel(host(bb), bo) < 1e-10
    acc.reset()
    acc.add_host(torch.from_numpy(x).pin_memory(), torch.from_numpy(y).pin_memory(), chunk=4096)
    T2, bb2, ntot2 = acc.system()
    acc.close()
    assert ntot2 == n
    assert rel(host(T2), To) < 1e-10
    assert rel(host(bb2), bo) < 1e-10


def test_host_fit_equals_device_fit():
    n, m, s, lam = 20011, 8, 2.0, 1e-4
    x, y = sample(2, n)
    xh = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).pin_memory()
    yh = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).pin_memory()
    a1 = fk.Accumulator(2, m, 1, 1e-6, "mixed")
    a1.add_host(xh, yh, chunk=3000)
    th_h = host(a1.fit_sobolev(s, [lam]))
    a1.close()
    a2 = fk.Accumulator(2, m, 1, 1e-6, "mixed")
    a2.add(xh.cuda(), yh.cuda())
    th_d = host(a2.fit_sobolev(s, [lam]))
    a2.close()
    assert rel(th_h, th_d) < 1e-6
    tho = O.fit(x.astype(np.float64), y[0].astype(np.float64), m, O.penalty_sobolev(2, m, lam, s))
    assert rel(th_h[0, 0], tho) < 1e-5


def test_host_argument_errors():
    acc = fk.Accumulator(2, 8, 1, 1e-6, "mixed")
    L = fk.lib()
    xh = torch.zeros((2, 10), dtype=torch.float32)
    yh = torch.zeros((1, 10), dtype=torch.float32)
    assert L.fk_accum_add_host(acc._h, 10, xh.data_ptr(), yh.data_ptr(), -1, None) == 1  # FK_EINVAL
    assert b"chunk" in L.fk_last_error()
    assert L.fk_accum_add_host(acc._h, 10, xh.data_ptr(), None, 0, None) == 1
    with pytest.raises(ValueError):
        acc.add_host(xh.double(), yh.double())
    with pytest.raises(ValueError):
        acc.add_host(xh.cuda(), yh)
    acc.close()
