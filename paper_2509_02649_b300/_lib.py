"""ctypes binding of libfk (include/fk.h): argument marshalling only.

Every function here takes torch tensors that already live on the GPU, checks
their dtype/layout, allocates the outputs with torch and passes raw device
pointers plus the current CUDA stream to the C-ABI.  All arithmetic runs in
libfk's kernels; there is no CPU fallback.  If libfk.so is missing the first
call raises.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np
import torch

from .build import lib_path

FK_FP64, FK_MIXED = 0, 1
FK_PEN_SOBOLEV, FK_PEN_LOWBIAS = 0, 1
FK_SOLVER_AUTO, FK_SOLVER_CHOL, FK_SOLVER_CG, FK_SOLVER_EIG = 0, 1, 2, 3
FK_SPREAD_AUTO, FK_SPREAD_ATOMIC, FK_SPREAD_BINNED, FK_SPREAD_FIXED, FK_SPREAD_FIXED_SHARED = 0, 1, 2, 3, 4

STATUS = {0: "FK_OK", 1: "FK_EINVAL", 2: "FK_ERANGE", 3: "FK_ENOMEM", 4: "FK_ECUDA", 5: "FK_ENOTPD",
          6: "FK_ENOCONV", 7: "FK_ETIMEOUT", 8: "FK_EINTERNAL"}

EXPORTS = ["fk_default_opts", "fk_fit_sobolev", "fk_fit_pik", "fk_fit_additive", "fk_predict", "fk_type1",
           "fk_type2", "fk_build_system", "fk_penalty_weights", "fk_solve", "fk_hypergrad", "fk_last_error",
           "fk_workspace_bytes", "fk_version", "fk_launch_count", "fk_type1_noalloc", "fk_penalty_grads",
           "fk_accum_create", "fk_accum_add", "fk_accum_system", "fk_accum_fit_sobolev", "fk_accum_reset",
           "fk_accum_destroy", "fk_generate_sweep_1d", "fk_release_workspace", "fk_autotune_table",
           "fk_autotune_clear", "fk_fit_pik_general", "fk_box_moments", "fk_fit_sobolev_pairs",
           "fk_capture_begin", "fk_capture_end", "fk_graph_launch", "fk_graph_status", "fk_graph_destroy",
           "fk_graph_kernel_ms", "fk_peak_fp32", "fk_peak_smem_atomics", "fk_accum_state_bytes", "fk_accum_save", "fk_accum_load",
           "fk_accum_add_state", "fk_heldout_loss", "fk_adjoint", "fk_accum_add_host"]


class FkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), msg))
        self.status = status
        self.name = STATUS.get(status, str(status))


class Opts(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("cg_tol", ctypes.c_double), ("cg_maxit", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("sobolev_c0", ctypes.c_double), ("upsampfac", ctypes.c_double),
                ("spread", ctypes.c_int), ("deterministic", ctypes.c_int), ("autotune", ctypes.c_int),
                ("wait_cycles", ctypes.c_longlong)]


class Report(ctypes.Structure):
    _fields_ = [("ms_spread", ctypes.c_double), ("ms_fft", ctypes.c_double), ("ms_solve", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("cg_iters", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("n_used", ctypes.c_int64), ("fine_grid", ctypes.c_int), ("kernel_width", ctypes.c_int),
                ("ms_kernel", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib: Optional[ctypes.CDLL] = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_int64
_D = ctypes.c_double


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("%s is not built (run paper_2509_02649_b300/build.py); no fallback exists"
                               % os.path.basename(path))
        L = ctypes.CDLL(path)
        sig = {
            "fk_default_opts": (None, [_P]),
            "fk_fit_sobolev": (_I, [_I, _L, _P, _P, _I, _I, _D, _I, _P, _I, _D, _I, _P, _P, _P, _P]),
            "fk_fit_pik": (_I, [_I, _L, _P, _P, _I, _I, _D, _D, _D, _I, _P, _P, _D, _I, _P, _P, _P, _P]),
            "fk_fit_additive": (_I, [_I, _L, _P, _P, _I, _I, _P, _I, _D, _I, _P, _P, _P, _P]),
            "fk_predict": (_I, [_I, _I, _I, _P, _I, _L, _P, _D, _I, _P, _P]),
            "fk_type1": (_I, [_I, _L, _P, _P, _I, _I, _D, _I, _P, _P]),
            "fk_type2": (_I, [_I, _I, _P, _I, _L, _P, _D, _I, _P, _P]),
            "fk_build_system": (_I, [_I, _L, _P, _P, _I, _I, _D, _I, _P, _P, _P, _P, _P]),
            "fk_penalty_weights": (_I, [_I, _I, _I, _D, _D, _P, _I, _D, _I, _P, _P, _P, _P]),
            "fk_solve": (_I, [_I, _I, _P, _P, _I, _P, _I, _P, _P, _P, _P]),
            "fk_hypergrad": (_I, [_I, _L, _P, _L, _P, _P, _I, _P, _P, _P, _D, _I, _P, _P, _P, _P, _P]),
            "fk_last_error": (ctypes.c_char_p, []),
            "fk_workspace_bytes": (ctypes.c_size_t, [_I, _I, _L, _I, _D, _I]),
            "fk_version": (ctypes.c_char_p, []),
            "fk_launch_count": (ctypes.c_int64, []),
            "fk_type1_noalloc": (_I, [_I, _L, _P, _P, _I, _I, _D, _I, _P, _P]),
            "fk_penalty_grads": (_I, [_I, _I, _D, _D, _D, _D, _I, _P, _P, _P, _P, _P]),
            "fk_accum_create": (_I, [_I, _I, _I, _D, _I, _P, ctypes.POINTER(_P), _P]),
            "fk_accum_add": (_I, [_P, _L, _P, _P, _P, _P]),
            "fk_accum_add_host": (_I, [_P, _L, _P, _P, _L, _P]),
            "fk_accum_system": (_I, [_P, _P, _P, ctypes.POINTER(_L), _P]),
            "fk_accum_fit_sobolev": (_I, [_P, _D, _I, _P, _I, _P, _P, _P]),
            "fk_accum_reset": (_I, [_P, _P]),
            "fk_accum_destroy": (_I, [_P]),
            "fk_generate_sweep_1d": (_I, [ctypes.c_uint64, _I, _L, _L, _I, _P, _P, _P, _P]),
            "fk_release_workspace": (_I, []),
            "fk_autotune_table": (ctypes.c_size_t, [ctypes.c_char_p, ctypes.c_size_t]),
            "fk_autotune_clear": (None, []),
            "fk_fit_pik_general": (_I, [_I, _L, _P, _P, _I, _I, _D, _D, _D, _I, _P, _P, _P, _D, _I, _P, _P, _P, _P]),
            "fk_box_moments": (_I, [_I, _I, _P, _P, _P, _P]),
            "fk_capture_begin": (_I, [_P]),
            "fk_capture_end": (_I, [_P, ctypes.POINTER(_P)]),
            "fk_graph_launch": (_I, [_P, _P]),
            "fk_graph_status": (_I, [_P]),
            "fk_graph_destroy": (_I, [_P]),
            "fk_graph_kernel_ms": (_I, [_P, ctypes.POINTER(ctypes.c_float)]),
            "fk_fit_sobolev_pairs": (_I, [_I, _L, _P, _P, _I, _I, _P, _P, _I, _I, _D, _I, _P, _P, _P, _P]),
            "fk_peak_fp32": (_I, [ctypes.POINTER(_D), ctypes.POINTER(_I), _P]),
            "fk_peak_smem_atomics": (_I, [ctypes.POINTER(_D), ctypes.POINTER(_D), _P]),
            "fk_accum_state_bytes": (ctypes.c_size_t, [_P]),
            "fk_accum_save": (_I, [_P, _P, ctypes.c_size_t, _P]),
            "fk_accum_load": (_I, [_P, _P, ctypes.c_size_t, _P]),
            "fk_accum_add_state": (_I, [_P, _P, ctypes.c_size_t, _P]),
            "fk_heldout_loss": (_I, [_I, _I, _P, _L, _P, _P, _D, _I, _P, _P, _P, _P]),
            "fk_adjoint": (_I, [_I, _I, _L, _P, _P, _P, _P, _P, _D, _I, _P, _D, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise FkError(status, lib().fk_last_error().decode())


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _prec(precision) -> int:
    if isinstance(precision, int):
        return precision
    return {"fp64": FK_FP64, "mixed": FK_MIXED}[precision]


_CAP = threading.local()


def _capturing() -> bool:
    return getattr(_CAP, "active", False)


def _dense(t: torch.Tensor) -> torch.Tensor:
    """t itself when contiguous; a copy otherwise, which a capture cannot record."""
    if t.is_contiguous():
        return t
    if _capturing():
        raise ValueError("inputs of a captured call must be contiguous (a copy would not outlive the capture)")
    return t.contiguous()


def _out(out, shape, dtype, device):
    if out is None:
        if _capturing():
            raise ValueError("pass out= to a captured call: its outputs must outlive the capture")
        return torch.empty(shape, dtype=dtype, device=device)
    if tuple(out.shape) != tuple(shape) or out.dtype != dtype or not out.is_contiguous() or out.device != device:
        raise ValueError("out must be a contiguous %s tensor of shape %s on %s" % (dtype, tuple(shape), device))
    return out


def _points(x: torch.Tensor, prec: int) -> torch.Tensor:
    want = torch.float64 if prec == FK_FP64 else torch.float32
    if not x.is_cuda:
        raise ValueError("points must be a CUDA tensor")
    if x.dtype != want:
        raise ValueError("points must be %s for this precision" % want)
    if x.dim() == 1:
        x = x.unsqueeze(0)
    return _dense(x)


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().fk_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _opts_ptr(opts):
    return ctypes.byref(opts) if opts is not None else None


def _dbl_array(vals: Sequence[float]):
    arr = (ctypes.c_double * len(vals))(*[float(v) for v in vals])
    return arr


def fk_build_system(x, y, m: int, eps: float, precision="mixed", opts: Optional[Opts] = None, report: bool = False,
                    out=None):
    """Moments T ((4m+1)^d complex) and right-hand sides b ([n_targets][D] complex), both / n.
    out: optional (T, b) tensors to write into (required during a capture)."""
    p = _prec(precision)
    x = _points(x, p)
    d, n = x.shape
    y = _dense(y.reshape(-1, n)) if y is not None else None
    nt = 0 if y is None else y.shape[0]
    T = _out(None if out is None else out[0], ((4 * m + 1) ** d,), torch.complex128, x.device)
    b = _out(None if out is None else out[1], (max(nt, 1), (2 * m + 1) ** d), torch.complex128, x.device)
    rep = Report()
    _check(lib().fk_build_system(d, n, x.data_ptr(), y.data_ptr() if y is not None else None, nt, m, eps, p,
                                 _opts_ptr(opts), T.data_ptr(), b.data_ptr(), _stream(),
                                 ctypes.byref(rep) if report else None))
    out = (T, b[:nt])
    return (out + (rep.as_dict(),)) if report else out


def fk_fit_sobolev(x, y, m: int, s: float, lambdas, eps: float, precision="mixed", penalty: int = FK_PEN_SOBOLEV,
                   opts: Optional[Opts] = None, report: bool = False, out=None):
    """theta [n_lambda][n_targets][D] complex128 (Eq. 2 with the Sec. 3.1 / 3.2 penalty)."""
    p = _prec(precision)
    x = _points(x, p)
    d, n = x.shape
    y = _dense(y.reshape(-1, n))
    lam = list(lambdas) if hasattr(lambdas, "__len__") else [lambdas]
    theta = _out(out, (len(lam), y.shape[0], (2 * m + 1) ** d), torch.complex128, x.device)
    rep = Report()
    _check(lib().fk_fit_sobolev(d, n, x.data_ptr(), y.data_ptr(), y.shape[0], m, s, penalty, _dbl_array(lam), len(lam),
                                eps, p, _opts_ptr(opts), theta.data_ptr(), _stream(),
                                ctypes.byref(rep) if report else None))
    return (theta, rep.as_dict()) if report else theta


def fk_fit_pik(x, y, m: int, s: float, lam: float, mu: float, alpha, a, eps: float, precision="mixed",
               opts: Optional[Opts] = None, report: bool = False):
    """theta [n_targets][D] complex128 with W = lambda(c0 + |k|^{2s}) + mu |P(ik)|^2 (Sec. 4)."""
    p = _prec(precision)
    x = _points(x, p)
    d, n = x.shape
    y = y.reshape(-1, n).contiguous()
    al = [int(v) for row in alpha for v in row]
    nt = len(a)
    alpha_arr = (ctypes.c_int * max(len(al), 1))(*al)
    theta = torch.empty((y.shape[0], (2 * m + 1) ** d), dtype=torch.complex128, device=x.device)
    rep = Report()
    _check(lib().fk_fit_pik(d, n, x.data_ptr(), y.data_ptr(), y.shape[0], m, s, lam, mu, nt, alpha_arr,
                            _dbl_array(a), eps, p, _opts_ptr(opts), theta.data_ptr(), _stream(),
                            ctypes.byref(rep) if report else None))
    return (theta, rep.as_dict()) if report else theta


def fk_fit_additive(x, y, m: int, lambdas, eps: float, precision="mixed", opts: Optional[Opts] = None,
                    report: bool = False, out=None):
    """theta [n_lambda][n_targets][d][2m+1] complex128 (Prop. 5.1)."""
    p = _prec(precision)
    x = _points(x, p)
    d, n = x.shape
    y = _dense(y.reshape(-1, n))
    lam = list(lambdas) if hasattr(lambdas, "__len__") else [lambdas]
    theta = _out(out, (len(lam), y.shape[0], d, 2 * m + 1), torch.complex128, x.device)
    rep = Report()
    _check(lib().fk_fit_additive(d, n, x.data_ptr(), y.data_ptr(), y.shape[0], m, _dbl_array(lam), len(lam), eps, p,
                                 _opts_ptr(opts), theta.data_ptr(), _stream(), ctypes.byref(rep) if report else None))
    return (theta, rep.as_dict()) if report else theta


def fk_predict(theta, xq, m: int, eps: float, precision="mixed", additive: bool = False, out=None):
    """f [n_sets][n_q] float64: Re sum_k theta_k e^{i<k,x>} (or the additive sum)."""
    p = _prec(precision)
    xq = _points(xq, p)
    d, nq = xq.shape
    per = d * (2 * m + 1) if additive else (2 * m + 1) ** d
    th = _dense(theta.reshape(-1, per))
    f = _out(out, (th.shape[0], nq), torch.float64, xq.device)
    _check(lib().fk_predict(1 if additive else 0, d, m, th.data_ptr(), th.shape[0], nq, xq.data_ptr(), eps, p,
                            f.data_ptr(), _stream()))
    return f


def fk_type1(x, c, kmax: int, eps: float, precision="mixed"):
    """Unnormalised sums out[c][k] = sum_i c_i e^{-i<k,x_i>} (complex128)."""
    p = _prec(precision)
    x = _points(x, p)
    d, n = x.shape
    c = c.reshape(-1, n).contiguous()
    out = torch.empty((c.shape[0], (2 * kmax + 1) ** d), dtype=torch.complex128, device=x.device)
    _check(lib().fk_type1(d, n, x.data_ptr(), c.data_ptr(), c.shape[0], kmax, eps, p, out.data_ptr(), _stream()))
    return out


def fk_type2(coef, x, kmax: int, eps: float, precision="mixed"):
    """Re sum_k coef_k e^{+i<k,x>} for each coefficient set, float64 [n_sets][n]."""
    p = _prec(precision)
    x = _points(x, p)
    d, n = x.shape
    cf = coef.reshape(-1, (2 * kmax + 1) ** d).contiguous()
    out = torch.empty((cf.shape[0], n), dtype=torch.float64, device=x.device)
    _check(lib().fk_type2(d, kmax, cf.data_ptr(), cf.shape[0], n, x.data_ptr(), eps, p, out.data_ptr(), _stream()))
    return out


def fk_penalty_weights(d: int, m: int, lambdas, s: float = 1.0, penalty: int = FK_PEN_SOBOLEV, c0: float = 1.0,
                       mu: float = 0.0, alpha=(), a=(), device="cuda"):
    lam = list(lambdas) if hasattr(lambdas, "__len__") else [lambdas]
    al = [int(v) for row in alpha for v in row]
    W = torch.empty((len(lam), (2 * m + 1) ** d), dtype=torch.float64, device=device)
    alpha_arr = (ctypes.c_int * max(len(al), 1))(*al)
    a_arr = _dbl_array(list(a) if len(a) else [0.0])
    _check(lib().fk_penalty_weights(d, m, penalty, s, c0, _dbl_array(lam), len(lam), mu, len(a), alpha_arr, a_arr,
                                    W.data_ptr(), _stream()))
    return W


def fk_solve(T, W, rhs, d: int, m: int, opts: Optional[Opts] = None, report: bool = False):
    """sol [n_w][n_rhs][D] complex128 of (Toep(T) + diag W_l) sol = rhs_r."""
    D = (2 * m + 1) ** d
    T = T.contiguous()
    W = W.reshape(-1, D).contiguous()
    rhs = rhs.reshape(-1, D).contiguous()
    sol = torch.empty((W.shape[0], rhs.shape[0], D), dtype=torch.complex128, device=T.device)
    rep = Report()
    _check(lib().fk_solve(d, m, T.data_ptr(), W.data_ptr(), W.shape[0], rhs.data_ptr(), rhs.shape[0],
                          _opts_ptr(opts), sol.data_ptr(), _stream(), ctypes.byref(rep) if report else None))
    return (sol, rep.as_dict()) if report else sol


def fk_hypergrad(x, xv, yv, m: int, T, W, theta, eps: float, precision="mixed", opts: Optional[Opts] = None,
                 want_dy: bool = True):
    """(loss, dL/dW [D] float64, dL/dY [n] float64 or None) by the adjoint method."""
    p = _prec(precision)
    x = _points(x, p)
    xv = _points(xv, p)
    d, n = x.shape
    nv = xv.shape[1]
    D = (2 * m + 1) ** d
    dW = torch.empty(D, dtype=torch.float64, device=x.device)
    dY = torch.empty(n, dtype=torch.float64, device=x.device) if want_dy else None
    loss = ctypes.c_double(0.0)
    _check(lib().fk_hypergrad(d, n, x.data_ptr(), nv, xv.data_ptr(), yv.contiguous().data_ptr(), m,
                              T.contiguous().data_ptr(), W.contiguous().data_ptr(), theta.contiguous().data_ptr(),
                              eps, p, _opts_ptr(opts), ctypes.byref(loss), dW.data_ptr(),
                              dY.data_ptr() if dY is not None else None, _stream()))
    return loss.value, dW, dY


def fk_peak_fp32():
    """(measured FP32 FMA throughput in TFLOP/s, multiprocessor count) of the current device."""
    t = _D()
    sms = _I()
    _check(lib().fk_peak_fp32(ctypes.byref(t), ctypes.byref(sms), _stream()))
    return t.value, sms.value


def fk_peak_smem_atomics():
    """(distinct-bank, random-window) throughput of 32-bit shared-memory atomic adds with a
    returned value, in 1e9 lane operations per second, on the current device."""
    dd = _D()
    dr = _D()
    _check(lib().fk_peak_smem_atomics(ctypes.byref(dd), ctypes.byref(dr), _stream()))
    return dd.value, dr.value


def fk_heldout_loss(theta, xv, yv, m: int, eps: float, precision="mixed", opts: Optional[Opts] = None):
    """(L = mean(r^2), r = f(xv) - yv on the device) for the fit theta (D complex)."""
    p = _prec(precision)
    xv = _points(xv, p)
    d, nv = xv.shape
    r = torch.empty(nv, dtype=xv.dtype, device=xv.device)
    loss = ctypes.c_double(0.0)
    _check(lib().fk_heldout_loss(d, m, _dense(theta).data_ptr(), nv, xv.data_ptr(), _dense(yv).data_ptr(), eps, p,
                                 _opts_ptr(opts), ctypes.byref(loss), r.data_ptr(), _stream()))
    return loss.value, r


def fk_adjoint(xv, r, T, W, theta, m: int, eps: float, precision="mixed", opts: Optional[Opts] = None,
               zscale: float = 0.0, want_zy: bool = False):
    """(dL/dW [D] float64, zy = zscale z [D] complex128 or None) from the residual r at xv."""
    p = _prec(precision)
    xv = _points(xv, p)
    d, nv = xv.shape
    D = (2 * m + 1) ** d
    dW = torch.empty(D, dtype=torch.float64, device=xv.device)
    zy = torch.empty(D, dtype=torch.complex128, device=xv.device) if want_zy else None
    _check(lib().fk_adjoint(d, m, nv, xv.data_ptr(), _dense(r).data_ptr(), _dense(T).data_ptr(), _dense(W).data_ptr(),
                            _dense(theta).data_ptr(), eps, p, _opts_ptr(opts), zscale, dW.data_ptr(),
                            zy.data_ptr() if zy is not None else None, _stream()))
    return dW, zy


def fk_launch_count() -> int:
    """Kernels libfk has launched in this process so far."""
    return int(lib().fk_launch_count())


def fk_type1_noalloc(x, c, kmax: int, eps: float, precision="mixed"):
    """fk_type1 through the entry point that allocates no device scratch (it uses the
    library's built-in scratch array); the output tensor is allocated here by torch."""
    p = _prec(precision)
    x = _points(x, p)
    d, n = x.shape
    c = c.reshape(-1, n).contiguous()
    out = torch.empty((c.shape[0], (2 * kmax + 1) ** d), dtype=torch.complex128, device=x.device)
    _check(lib().fk_type1_noalloc(d, n, x.data_ptr(), c.data_ptr(), c.shape[0], kmax, eps, p, out.data_ptr(),
                                  _stream()))
    return out


def fk_penalty_grads(d: int, m: int, dW, lam: float, s: float = 1.0, mu: float = 0.0, alpha=(), a=(), c0: float = 1.0):
    """[dL/dlambda, dL/ds, dL/dmu, dL/da_0, ...] (host floats) from dL/dW (device)."""
    al = [int(v) for row in alpha for v in row]
    alpha_arr = (ctypes.c_int * max(len(al), 1))(*al)
    a_arr = _dbl_array(list(a) if len(a) else [0.0])
    out = (ctypes.c_double * (3 + len(a)))()
    _check(lib().fk_penalty_grads(d, m, s, c0, lam, mu, len(a), alpha_arr, a_arr, dW.contiguous().data_ptr(), out,
                                  _stream()))
    return list(out)


class Accumulator:
    """Streaming sums of T and b over chunks of points (fk_accum_*): add chunks with
    add(), then system() or fit_sobolev().  The device grids are freed by close()."""

    def __init__(self, d: int, m: int, n_targets: int, eps: float, precision="mixed",
                 opts: Optional[Opts] = None, device=None):
        self.d, self.m, self.nt = d, m, n_targets
        self.prec = _prec(precision)
        self.device = torch.device("cuda") if device is None else torch.device(device)
        h = _P()
        _check(lib().fk_accum_create(d, m, n_targets, eps, self.prec, _opts_ptr(opts), ctypes.byref(h), _stream()))
        self._h = h
        self._keep = []  # chunk tensors kept alive until the next synchronising call

    def add(self, x, y=None, y_absmax=None, keep: bool = True):
        """Spread a chunk.  keep=False drops the references to the chunk at once: safe when
        its memory comes from torch on the current stream, whose caching allocator hands
        it out again only to work ordered after this call."""
        x = _points(x, self.prec)
        n = x.shape[1]
        if x.shape[0] != self.d:
            raise ValueError("points have %d coordinates, accumulator %d" % (x.shape[0], self.d))
        if self.nt:
            y = y.reshape(self.nt, n).contiguous()
        if y_absmax is not None and y_absmax.dtype != torch.int32:
            raise ValueError("y_absmax must be the int32 bit patterns written by generate_sweep_1d")
        _check(lib().fk_accum_add(self._h, n, x.data_ptr(), y.data_ptr() if self.nt else None,
                                  y_absmax.data_ptr() if y_absmax is not None else None, _stream()))
        if keep:
            self._keep.append((x, y, y_absmax))

    def add_host(self, x, y=None, chunk: int = 0):
        """Spread points held in host memory (fk_accum_add_host): x (d, n) and y
        (n_targets, n) CPU tensors of the accumulator's dtype, page-locked for the link's
        full rate.  They are kept alive until the next synchronising call."""
        dt = torch.float64 if self.prec == FK_FP64 else torch.float32
        if x.device.type != "cpu" or x.dtype != dt or x.dim() != 2 or x.shape[0] != self.d:
            raise ValueError("x must be a CPU tensor of shape (%d, n) and dtype %s" % (self.d, dt))
        x = x.contiguous()
        n = x.shape[1]
        if self.nt:
            if y is None or y.device.type != "cpu" or y.dtype != dt or y.numel() != self.nt * n:
                raise ValueError("y must be a CPU tensor of %d x %d values of dtype %s" % (self.nt, n, dt))
            y = y.reshape(self.nt, n).contiguous()
        _check(lib().fk_accum_add_host(self._h, n, x.data_ptr(), y.data_ptr() if self.nt else None, int(chunk),
                                       _stream()))
        self._keep.append((x, y))

    def system(self):
        T = torch.empty((4 * self.m + 1) ** self.d, dtype=torch.complex128, device=self.device)
        b = torch.empty((max(self.nt, 1), (2 * self.m + 1) ** self.d), dtype=torch.complex128, device=self.device)
        nt = _L()
        _check(lib().fk_accum_system(self._h, T.data_ptr(), b.data_ptr() if self.nt else None, ctypes.byref(nt),
                                     _stream()))
        self._keep.clear()
        return T, b[:self.nt], int(nt.value)

    def fit_sobolev(self, s: float, lambdas, penalty: int = FK_PEN_SOBOLEV, report: bool = False):
        lam = list(lambdas) if hasattr(lambdas, "__len__") else [lambdas]
        theta = torch.empty((len(lam), self.nt, (2 * self.m + 1) ** self.d), dtype=torch.complex128,
                            device=self.device)
        rep = Report()
        _check(lib().fk_accum_fit_sobolev(self._h, s, penalty, _dbl_array(lam), len(lam), theta.data_ptr(), _stream(),
                                          ctypes.byref(rep) if report else None))
        self._keep.clear()
        return (theta, rep.as_dict()) if report else theta

    def reset(self):
        _check(lib().fk_accum_reset(self._h, _stream()))

    def state(self) -> bytes:
        """The sums so far (point count, device flags, fp64 grids) as bytes: a checkpoint,
        or one shard's part of a reduction."""
        n = int(lib().fk_accum_state_bytes(self._h))
        buf = ctypes.create_string_buffer(n)
        _check(lib().fk_accum_save(self._h, buf, n, _stream()))
        return buf.raw

    def load_state(self, state: bytes):
        """Replace the sums by a saved state (same accumulator shape)."""
        _check(lib().fk_accum_load(self._h, state, len(state), _stream()))

    def add_state(self, state: bytes):
        """Add another accumulator's saved sums (shard reduction)."""
        _check(lib().fk_accum_add_state(self._h, state, len(state), _stream()))

    def close(self):
        if self._h:
            torch.cuda.current_stream().synchronize()
            _check(lib().fk_accum_destroy(self._h))
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate_sweep_1d(first: int, n: int, n_targets: int = 16, seed: int = 20250902, workload: int = 5,
                      out=None, device=None):
    """Points first .. first + n - 1 of the counter-based 1-D sweep sample (device):
    returns x (1, n) float32, y (n_targets, n) float32 and max|y_t| as int32 float bits."""
    dev = torch.device("cuda") if device is None else torch.device(device)
    if out is None:
        x = torch.empty((1, n), dtype=torch.float32, device=dev)
        y = torch.empty((n_targets, n), dtype=torch.float32, device=dev)
        amax = torch.empty(max(n_targets, 1), dtype=torch.int32, device=dev)
    else:
        x, y, amax = out
        if not (x.is_contiguous() and y.is_contiguous() and x.numel() == n and y.shape == (n_targets, n)
                and x.dtype == torch.float32 and y.dtype == torch.float32 and amax.dtype == torch.int32
                and amax.numel() >= n_targets):
            raise ValueError("out must be contiguous float32 x (1, n), y (n_targets, n) and int32 amax")
    _check(lib().fk_generate_sweep_1d(seed, workload, first, n, n_targets, x.data_ptr(), y.data_ptr(),
                                      amax.data_ptr(), _stream()))
    return x, y, amax


def fk_release_workspace():
    """Return the library's unused workspace memory on the current device."""
    _check(lib().fk_release_workspace())


def fk_autotune_table() -> str:
    """The tuned problem classes and their measured shapes, one line each."""
    need = lib().fk_autotune_table(None, 0)
    buf = ctypes.create_string_buffer(int(need))
    lib().fk_autotune_table(buf, need)
    return buf.value.decode()


def fk_autotune_clear():
    lib().fk_autotune_clear()


def fk_box_moments(d: int, m: int, lo, hi, device=None):
    """c_j = (2 pi)^{-d} int_box e^{-i<j,x>} dx, |j|_inf <= 2m (device complex128)."""
    dev = torch.device("cuda") if device is None else torch.device(device)
    c = torch.empty((4 * m + 1) ** d, dtype=torch.complex128, device=dev)
    lo_a = _dbl_array([float(v) for v in np.broadcast_to(np.asarray(lo, dtype=float), (d,))])
    hi_a = _dbl_array([float(v) for v in np.broadcast_to(np.asarray(hi, dtype=float), (d,))])
    _check(lib().fk_box_moments(d, m, lo_a, hi_a, c.data_ptr(), _stream()))
    return c


def fk_fit_pik_general(x, y, m: int, s: float, lam: float, mu: float, alpha, a, c_moments, eps: float,
                       precision="mixed", opts: Optional[Opts] = None, report: bool = False):
    """theta [n_targets][D] with the penalty lambda(c0 + |k|^{2s}) + mu D^* C D, C = Toep(c_moments)."""
    p = _prec(precision)
    x = _points(x, p)
    d, n = x.shape
    y = y.reshape(-1, n).contiguous()
    al = [int(v) for row in alpha for v in row]
    alpha_arr = (ctypes.c_int * max(len(al), 1))(*al)
    theta = torch.empty((y.shape[0], (2 * m + 1) ** d), dtype=torch.complex128, device=x.device)
    c = c_moments.contiguous()
    rep = Report()
    _check(lib().fk_fit_pik_general(d, n, x.data_ptr(), y.data_ptr(), y.shape[0], m, s, lam, mu, len(a), alpha_arr,
                                    _dbl_array(a), c.data_ptr(), eps, p, _opts_ptr(opts), theta.data_ptr(), _stream(),
                                    ctypes.byref(rep) if report else None))
    return (theta, rep.as_dict()) if report else theta


def fk_fit_sobolev_pairs(x, y, m: int, s_values, lambdas, eps: float, precision="mixed",
                         penalty: int = FK_PEN_SOBOLEV, opts: Optional[Opts] = None, report: bool = False):
    """theta [n_pairs][n_targets][D]: one fit per (s_i, lambda_i) from one spreading pass."""
    p = _prec(precision)
    x = _points(x, p)
    d, n = x.shape
    y = y.reshape(-1, n).contiguous()
    sv, lv = [float(v) for v in s_values], [float(v) for v in lambdas]
    if len(sv) != len(lv):
        raise ValueError("s_values and lambdas differ in length")
    theta = torch.empty((len(sv), y.shape[0], (2 * m + 1) ** d), dtype=torch.complex128, device=x.device)
    rep = Report()
    _check(lib().fk_fit_sobolev_pairs(d, n, x.data_ptr(), y.data_ptr(), y.shape[0], m, _dbl_array(sv), _dbl_array(lv),
                                      len(sv), penalty, eps, p, _opts_ptr(opts), theta.data_ptr(), _stream(),
                                      ctypes.byref(rep) if report else None))
    return (theta, rep.as_dict()) if report else theta


class Graph:
    """Library calls recorded by `capture`, replayed with one graph launch."""

    def __init__(self):
        self._ptr = _P()

    def launch(self, stream=None):
        if not self._ptr:
            raise ValueError("graph is closed or was not captured")
        _check(lib().fk_graph_launch(self._ptr, _stream(stream)))

    def status(self):
        """Waits for the last launch and raises FkError on a device-side condition."""
        _check(lib().fk_graph_status(self._ptr))

    def kernel_ms(self) -> float:
        """Time of the main spreading kernel in the last launch (event record nodes)."""
        v = ctypes.c_float()
        _check(lib().fk_graph_kernel_ms(self._ptr, ctypes.byref(v)))
        return v.value

    def close(self):
        if self._ptr:
            lib().fk_graph_destroy(self._ptr)
            self._ptr = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@contextlib.contextmanager
def capture(stream=None):
    """Record the library calls of the block (made on `stream`, which becomes the current
    stream inside) into a Graph.  Calls inside record work only; pass out= for their
    outputs and keep inputs and outputs alive while the graph is used."""
    s = torch.cuda.Stream() if stream is None else stream
    if s.cuda_stream == 0:
        raise ValueError("capture needs a created stream, not the default stream")
    g = Graph()
    g.stream = s
    s.wait_stream(torch.cuda.current_stream())
    _check(lib().fk_capture_begin(s.cuda_stream))
    _CAP.active = True
    ok = False
    try:
        with torch.cuda.stream(s):
            yield g
        ok = True
    finally:
        _CAP.active = False
        rc = lib().fk_capture_end(s.cuda_stream, ctypes.byref(g._ptr))
        if ok:
            _check(rc)
