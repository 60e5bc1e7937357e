"""The allocation-free reduction entry point (dwf_norm2_noalloc) against the
allocating one (dwf_norm2), through the C ABI.

dwf_norm2_noalloc exists for callers that cannot call cudaMalloc when they
need a global sum (for example code running under a memory pool that forbids
new allocations, or a plug-in handed only its input and output buffers): its
scratch is a static device array inside the library, so the call allocates
nothing.  This file is collected last so that a failure here does not hide
the other GPU tests in a run that stops at the first failure."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from paper_2103_05034_gb300 import _lib, layout, ops
from paper_2103_05034_gb300._lib import DWF_EINVAL, F16S, F32, F64

pytestmark = pytest.mark.gpu


def _call(a, n, prec):
    r = C.c_double(-1.0)
    code = _lib.lib().dwf_norm2_noalloc(C.byref(r), C.c_void_p(a.data_ptr()), n, prec,
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, r.value


@pytest.mark.parametrize("prec", [F64, F32, F16S])
def test_noalloc_norm2_matches_allocating_entry_point(prec):
    L, Ls = (4, 4, 4, 8), 8
    ctx = ops.Context(L, Ls, 1.8, synth.random_gauge(L, 0.3, 3))
    big = torch.from_numpy(layout.complex_to_real(
        layout.to_full(synth.gaussian_spinor(L, Ls, 91), L), prec).reshape(-1)).cuda()
    small = big[: big.numel() // 3 // 2 * 2].clone()
    # FP64 data: both sum the squares in FP64, in different orders.  FP32
    # and FP16-storage data (the same half values read by both): the
    # allocating reduction accumulates each thread's share in compensated
    # FP32 (a few ulp of FP32, 1e-7 relative at most) and the allocation-free
    # one in FP64.
    tol = 1e-12 if prec == F64 else 1e-6
    for a in (big, small):  # two calls in a row; the second sees the first's scratch contents
        n = a.numel() // 2
        ref = ops.dwf_norm2(ctx, a)
        code, got = _call(a, n, prec)
        assert code == 0
        assert abs(got - ref) <= tol * ref
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    a = torch.zeros(2, dtype=torch.float64, device="cuda")
    code, _ = _call(a, (1 << 31) + 1, F64)  # more than 2^31 complex numbers
    assert code == DWF_EINVAL
