"""fk_type1_noalloc: the type-1 transform for callers that cannot allocate device
memory at call time (their device memory is wholly reserved by their own pool
allocator, or their policy forbids allocation after start-up).  It takes its
scratch from a built-in device array instead of cudaMallocAsync.

The entry point is called through the C-ABI with outputs allocated beforehand.
Its results are checked against fk_type1 (the allocating entry point) and against
the CPU oracle on two calls in a row, with the tolerance the type-1 parity tests use
(10 * eps, normwise), and the device's free memory must not change across a call
after the first (set-up) call.  This file is collected last so that a run stopping
at its first failure has run every other test already; it also passes alone in a
fresh process.
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


def call_noalloc(x, c, kmax, eps, prec, out):
    """fk_type1_noalloc through the C-ABI; raises on a status other than FK_OK."""
    d, n = x.shape
    st = fk.lib().fk_type1_noalloc(d, n, x.data_ptr(), c.data_ptr(), c.shape[0], kmax, eps, prec, out.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    if st != 0:
        raise fk.FkError(st, fk.lib().fk_last_error().decode())


@pytest.mark.parametrize("precision,eps,dtype", [("fp64", 1e-12, torch.float64), ("mixed", 1e-6, torch.float32)])
@pytest.mark.parametrize("d,kmax,n", [(1, 60, 5003), (2, 16, 20011)])
def test_noalloc_matches_allocating_type1_and_oracle_twice(precision, eps, dtype, d, kmax, n):
    xh = S.uniform_points(n, d, 41)
    ch = np.stack([S.noise(n, 1.0, 41, 5), np.ones(n)])
    x = torch.from_numpy(xh).to("cuda", dtype).contiguous()
    c = torch.from_numpy(ch).to("cuda", dtype).contiguous()
    prec = fk.FK_FP64 if precision == "fp64" else fk.FK_MIXED
    ref = fk.fk_type1(x, c, kmax, eps, precision).cpu().numpy()
    # the oracle on the inputs as the GPU sees them (fp32-rounded in the mixed case)
    xo = x.double().cpu().numpy()
    co = c.double().cpu().numpy()
    orc = np.stack([O.type1(xo, co[k], kmax) for k in range(2)])
    out = torch.empty((2, (2 * kmax + 1) ** d), dtype=torch.complex128, device="cuda")
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out.zero_()
        call_noalloc(x, c, kmax, eps, prec, out)
        got = out.cpu().numpy()
        for k in range(2):
            assert rel(got[k], ref[k]) <= 10 * eps
            assert rel(got[k], orc[k]) <= 10 * eps


def test_noalloc_allocates_no_device_memory_after_setup():
    n, kmax, eps = 40000, 24, 1e-6
    x = torch.from_numpy(S.uniform_points(n, 2, 43)).to("cuda", torch.float32).contiguous()
    c = torch.ones((1, n), dtype=torch.float32, device="cuda")
    out = torch.empty((1, (2 * kmax + 1) ** 2), dtype=torch.complex128, device="cuda")
    call_noalloc(x, c, kmax, eps, fk.FK_MIXED, out)  # set-up on this device (if not done yet)
    first = out.clone()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        call_noalloc(x, c, kmax, eps, fk.FK_MIXED, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # the fp64 atomic sums may add in another order: equal to rounding
    assert float((out - first).abs().max() / first.abs().max()) <= 1e-12


def test_noalloc_rejects_shapes_beyond_its_scratch():
    x = torch.zeros((2, 16), dtype=torch.float32, device="cuda")
    c = torch.ones((8, 16), dtype=torch.float32, device="cuda")
    out = torch.empty((8, 601 ** 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(fk.FkError) as e:
        call_noalloc(x, c, 300, 1e-6, fk.FK_MIXED, out)  # 8 channels on a 2048^2 grid
    assert e.value.name == "FK_EINVAL" and "limit" in str(e.value)
