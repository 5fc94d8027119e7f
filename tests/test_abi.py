"""The C-ABI library loads, exports every symbol include/fk.h declares, and rejects
bad arguments on the host before touching the GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_2509_02649_b300 as fk
from paper_2509_02649_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^FK_API\s+[\w\s\*]+?\b(fk_\w+)\s*\(", src, re.M))
    return names


def test_library_exports_every_declared_symbol():
    L = fk.lib()
    names = declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    assert set(_lib.EXPORTS) == names


def test_checked_build_exports_the_same_symbols():
    """The bounds-checked build (FK_CHECKED) exports the same C-ABI."""
    path = os.path.join(ROOT, "paper_2509_02649_b300", "libfk_checked.so")
    if not os.path.exists(path):
        pytest.skip("libfk_checked.so is not built")
    L = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_version_and_defaults():
    L = fk.lib()
    assert b"sm_103a" in L.fk_version()
    o = fk.default_opts()
    assert o.cg_tol == 1e-13 and o.refine_steps == 1 and o.sobolev_c0 == 1.0


@pytest.mark.parametrize("args,needle", [
    (dict(d=5), b"d = 5"),
    (dict(n=0), b"n = 0"),
    (dict(m=-1), b"m = -1"),
    (dict(eps=1.0), b"eps"),
    (dict(lam=-1.0), b"lambda"),
    (dict(precision=7), b"precision"),
])
def test_invalid_arguments_rejected_on_host(args, needle):
    L = fk.lib()
    a = dict(d=1, n=10, m=3, eps=1e-6, lam=1e-3, precision=1)
    a.update(args)
    lam = (ctypes.c_double * 1)(a["lam"])
    dummy = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    st = L.fk_fit_sobolev(a["d"], a["n"], dummy, dummy, 1, a["m"], 1.0, 0, lam, 1, a["eps"], a["precision"],
                          None, dummy, None, None)
    assert st == 1  # FK_EINVAL
    assert needle in L.fk_last_error()


def test_workspace_bound_is_positive():
    assert fk.lib().fk_workspace_bytes(2, 32, 10 ** 8, 1, 1e-6, 1) > 0


def test_host_add_rejects_a_null_accumulator():
    L = fk.lib()
    dummy = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    assert L.fk_accum_add_host(None, 10, dummy, dummy, 0, None) == 1  # FK_EINVAL
    assert b"null accumulator" in L.fk_last_error()
