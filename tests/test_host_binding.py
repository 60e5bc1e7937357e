"""Host logic of the binding, without a GPU: the C-ABI entry points added for
the batched and baseline solvers reject a null context before any CUDA call,
the Python wrappers marshal per-system masses and statistics through ctypes,
turn a status code into an exception, and fail loudly when the library is
missing (there is no CPU fallback)."""
import ctypes

import numpy as np
import pytest

from paper_2103_05034_gb300 import _lib, ops


@pytest.fixture(scope="module")
def built():
    import os
    if not os.path.exists(_lib.LIB_PATH):
        import __graft_entry__ as g
        g.build()
    return _lib.lib()


def test_new_entry_points_reject_null_context(built):
    mf = (ctypes.c_double * 2)(0.01, 0.2)
    st = (_lib.SolveStats * 2)()
    for fn in (built.rbcg_solve_batch, built.rbcg_normal_solve_batch):
        assert fn(None, None, None, mf, 2, 1e-8, 10, _lib.SOLVE_F64, st, None) == _lib.DWF_EINVAL
    assert built.cgnr_solve(None, None, None, 0.01, 1e-8, 10, None, None) == _lib.DWF_EINVAL
    assert built.coarse_apply_status(None, None) == _lib.DWF_EINVAL


class _FakeLib:
    """Stands in for the loaded library: records the arguments of the batched
    solver and fills one statistics entry per system."""

    def __init__(self, code=0):
        self.code = code
        self.calls = []

    def rbcg_solve_batch(self, h, x, b, mf, n, tol, maxiter, policy, stats, stream):
        self.calls.append((h, [mf[i] for i in range(n)], n, tol, maxiter, policy))
        for i in range(n):
            stats[i].iterations = 100 + i
            stats[i].true_residual = 1e-9 * (i + 1)
        return self.code

    rbcg_normal_solve_batch = rbcg_solve_batch

    def dwf_last_error(self, h):
        return b"maxiter reached before tol"


class _Ctx:
    h = ctypes.c_void_p(1234)


def test_batch_wrappers_marshal_masses_and_stats(monkeypatch):
    fake = _FakeLib()
    monkeypatch.setattr(_lib, "_lib", fake)
    x = np.zeros(16)
    b = np.ones(16)
    st = ops.rbcg_solve_batch(_Ctx(), x, b, [0.01, 0.05, 0.2], 1e-8, 77, _lib.SOLVE_MIXED_F32)
    assert [s["iterations"] for s in st] == [100, 101, 102]
    assert st[2]["true_residual"] == pytest.approx(3e-9)
    _, masses, n, tol, maxiter, policy = fake.calls[0]
    assert masses == [0.01, 0.05, 0.2] and n == 3 and tol == 1e-8 and maxiter == 77
    assert policy == _lib.SOLVE_MIXED_F32
    st = ops.rbcg_normal_solve_batch(_Ctx(), x, b, [1.0], 1e-10)
    assert len(st) == 1 and fake.calls[1][1] == [1.0]


def test_status_code_raises(monkeypatch):
    monkeypatch.setattr(_lib, "_lib", _FakeLib(code=_lib.DWF_ENOCONV))
    with pytest.raises(_lib.DWFError) as e:
        ops.rbcg_solve_batch(_Ctx(), np.zeros(4), np.ones(4), [0.01], 1e-8)
    assert e.value.code == _lib.DWF_ENOCONV
    assert "maxiter" in str(e.value)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        ops.rbcg_solve_batch(_Ctx(), np.zeros(4), np.ones(4), [0.01], 1e-8)
