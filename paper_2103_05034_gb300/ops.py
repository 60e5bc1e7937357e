"""Python binding of the C ABI (include/dwfmg.h): argument marshalling only.

Every function takes torch tensors for field buffers (device tensors for the
operators, device or host tensors for the solvers) and runs on the current
torch CUDA stream.  Field tensors hold interleaved (re, im) reals of the
precision's type: float64 (DWF_F64), float32 (DWF_F32) or float16 (DWF_F16S),
laid out as documented in the header.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import F16S, F32, F64, SolveStats, check, lib

_DTYPE = {F64: torch.float64, F32: torch.float32, F16S: torch.float16}


def _stream():
    if torch.cuda.is_available():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(0)


def _ptr(t):
    if isinstance(t, np.ndarray):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(t.data_ptr())


def _prec_of(t):
    for p, dt in _DTYPE.items():
        if t.dtype == dt:
            return p
    raise TypeError(f"unsupported field dtype {t.dtype}")


class Context:
    """A dwf_ctx: lattice geometry, M5 and the gauge field (Sec. 2)."""

    def __init__(self, L, Ls, M5, gauge):
        g = gauge
        if isinstance(g, np.ndarray):
            g = np.ascontiguousarray(g, dtype=np.complex128)
        elif isinstance(g, torch.Tensor) and g.is_complex():
            g = torch.view_as_real(g.contiguous())
        self._gauge_ref = g
        h = C.c_void_p()
        Larr = (C.c_int * 4)(*L)
        check(lib().dwf_ctx_create(C.byref(h), Larr, int(Ls), float(M5), _ptr(g), _stream()))
        self.h = h
        self.L = tuple(L)
        self.Ls = Ls
        self.M5 = M5
        self.Vh = lib().dwf_half_sites(h)
        del self._gauge_ref

    def close(self):
        if getattr(self, "h", None):
            lib().dwf_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def half_numel(self):
        """Real numbers in one half field."""
        return self.Vh * 12 * self.Ls * 2

    def new_half(self, prec=F32, nrhs=1, device="cuda"):
        return torch.zeros(nrhs * self.half_numel(), dtype=_DTYPE[prec], device=device)

    def new_full(self, prec=F32, nrhs=1, device="cuda"):
        return torch.zeros(2 * nrhs * self.half_numel(), dtype=_DTYPE[prec], device=device)


def dwf_dhop(ctx, out, inp, out_parity, dagger=0, nrhs=1):
    check(lib().dwf_dhop(ctx.h, _ptr(out), _ptr(inp), out_parity, dagger, _prec_of(inp), nrhs,
                         _stream()), ctx.h)
    return out


def dwf_mooee(ctx, out, inp, mf, dagger=0, nrhs=1):
    check(lib().dwf_mooee(ctx.h, _ptr(out), _ptr(inp), mf, dagger, _prec_of(inp), nrhs, _stream()),
          ctx.h)
    return out


def dwf_mooee_inv(ctx, out, inp, mf, dagger=0, nrhs=1):
    check(lib().dwf_mooee_inv(ctx.h, _ptr(out), _ptr(inp), mf, dagger, _prec_of(inp), nrhs,
                              _stream()), ctx.h)
    return out


def dwf_mpc(ctx, out, inp, mf, dagger=0, nrhs=1):
    check(lib().dwf_mpc(ctx.h, _ptr(out), _ptr(inp), mf, dagger, _prec_of(inp), nrhs, _stream()),
          ctx.h)
    return out


def dwf_mpcdag_mpc(ctx, out, inp, mf, nrhs=1):
    check(lib().dwf_mpcdag_mpc(ctx.h, _ptr(out), _ptr(inp), mf, _prec_of(inp), nrhs, _stream()),
          ctx.h)
    return out


def dwf_ddw(ctx, out, inp, mf, dagger=0, nrhs=1):
    check(lib().dwf_ddw(ctx.h, _ptr(out), _ptr(inp), mf, dagger, _prec_of(inp), nrhs, _stream()),
          ctx.h)
    return out


def dwf_hdw(ctx, out, inp, mf, nrhs=1):
    check(lib().dwf_hdw(ctx.h, _ptr(out), _ptr(inp), mf, _prec_of(inp), nrhs, _stream()), ctx.h)
    return out


def dwf_norm2(ctx, a):
    r = C.c_double()
    check(lib().dwf_norm2(ctx.h, C.byref(r), _ptr(a), a.numel() // 2, _prec_of(a), _stream()), ctx.h)
    return r.value


def dwf_cdot(ctx, a, b):
    r = (C.c_double * 2)()
    check(lib().dwf_cdot(ctx.h, r, _ptr(a), _ptr(b), a.numel() // 2, _prec_of(a), _stream()), ctx.h)
    return complex(r[0], r[1])


def rbcg_solve(ctx, x, b, mf, tol, maxiter=100000, policy=_lib.SOLVE_MIXED_F32):
    """Red-black CGNR solve of D_DW x = b (full FP64 fields, host or device).
    Returns the solver statistics as a dict."""
    st = SolveStats()
    code = lib().rbcg_solve(ctx.h, _ptr(x), _ptr(b), mf, tol, maxiter, policy, C.byref(st),
                            _stream())
    check(code, ctx.h)
    return st.as_dict()


def dwf_power_max(ctx, v0, mf, iters):
    r = C.c_double()
    check(lib().dwf_power_max(ctx.h, C.byref(r), _ptr(v0), mf, iters, _stream()), ctx.h)
    return r.value
