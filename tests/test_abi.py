"""The C-ABI library loads and exports every function include/dwfmg.h declares
(no compute call: runs without a GPU), and the host layout marshalling
round-trips."""
import ctypes
import os

import numpy as np
import pytest

import synth
from paper_2103_05034_gb300 import _lib, layout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    return _lib.lib()


def test_library_exports_every_header_function(built):
    names = _lib.header_functions()
    assert len(names) >= 16
    raw = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert set(_lib.header_functions()) == set(_lib._SIGS)


def test_null_context_is_rejected_without_gpu(built):
    # argument validation happens before any CUDA call
    assert built.dwf_dhop(None, None, None, 0, 0, 1, 1, None) == _lib.DWF_EINVAL
    assert built.rbcg_solve(None, None, None, 0.01, 1e-8, 10, 1, None, None) == _lib.DWF_EINVAL
    bad = (ctypes.c_int * 4)(4, 4, 4, 5)
    h = ctypes.c_void_p()
    dummy = np.zeros(8)
    assert built.dwf_ctx_create(ctypes.byref(h), bad, 8, 1.8, dummy.ctypes.data, None) == _lib.DWF_EINVAL
    good = (ctypes.c_int * 4)(4, 4, 4, 4)
    assert built.dwf_ctx_create(ctypes.byref(h), good, 7, 1.8, dummy.ctypes.data, None) == _lib.DWF_EINVAL


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (2, 2, 2, 6), (6, 4, 2, 2)])
def test_layout_roundtrip(L):
    Ls = 4
    psi = synth.gaussian_spinor(L, Ls, 3)
    full = layout.to_full(psi, L)
    assert full.shape == (2, np.prod(L) // 2, 4, 3, Ls)
    assert np.array_equal(layout.from_full(full, L), psi)
    # even sites of the half field are the lexicographic even sites in order
    x = np.arange(np.prod(L)).reshape(L[::-1])
    par = layout.parity_of_lex(L)
    lex_even = np.where(par == 0)[0]
    assert np.array_equal(lex_even // 2, np.arange(len(lex_even)))
    r = layout.complex_to_real(full, 1)
    assert r.dtype == np.float32 and r.size == 2 * full.size


def test_header_constants_match_binding():
    import re
    text = open(os.path.join(ROOT, "include", "dwfmg.h")).read()
    consts = dict((k, int(v)) for k, v in re.findall(r"#define (DWF_\w+) (-?\d+)", text))
    assert consts["DWF_HOP_VARIANTS"] == _lib.HOP_VARIANTS
    assert (consts["DWF_F64"], consts["DWF_F32"], consts["DWF_F16S"], consts["DWF_TF32"]) == \
        (_lib.F64, _lib.F32, _lib.F16S, _lib.TF32)
