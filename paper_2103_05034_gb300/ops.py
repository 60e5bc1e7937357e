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
from ._lib import F16S, F32, F64, TF32, SolveStats, check, lib

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


def dwf_counters(ctx):
    """(kernel launches, algorithmic hopping-term bytes) since the last reset."""
    n = C.c_int64()
    b = C.c_double()
    check(lib().dwf_counters(ctx.h, C.byref(n), C.byref(b)))
    return n.value, b.value


def dwf_reset_counters(ctx):
    check(lib().dwf_reset_counters(ctx.h))


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


def rbcg_solve(ctx, x, b, mf, tol, maxiter=100000, policy=_lib.SOLVE_MIXED_F32, noconv_ok=False):
    """Red-black CGNR solve of D_DW x = b (full FP64 fields, host or device).
    Returns the solver statistics as a dict.  noconv_ok: a solve stopped by
    maxiter (DWF_ENOCONV, x still written) returns its statistics instead of
    raising."""
    st = SolveStats()
    code = lib().rbcg_solve(ctx.h, _ptr(x), _ptr(b), mf, tol, maxiter, policy, C.byref(st),
                            _stream())
    if not (noconv_ok and code == _lib.DWF_ENOCONV):
        check(code, ctx.h)
    return st.as_dict()


def rbcg2_solve(ctx, x, b, mf, tol, maxiter=100000, policy=_lib.SOLVE_F64):
    """Red-black CGNR with the second Schur form M_ee^-1 M_pc (Table 5);
    arguments and result as rbcg_solve."""
    st = SolveStats()
    check(lib().rbcg2_solve(ctx.h, _ptr(x), _ptr(b), mf, tol, maxiter, policy, C.byref(st), _stream()),
          ctx.h)
    return st.as_dict()


def dwf_power_max(ctx, v0, mf, iters, prec=F64):
    r = C.c_double()
    check(lib().dwf_power_max(ctx.h, C.byref(r), _ptr(v0), mf, iters, prec, _stream()), ctx.h)
    return r.value


# ---------------------------------------------------------------------- subspace and multigrid
def _ivec(v):
    return (C.c_int * 4)(*v)


def cheby_filter(ctx, out, inp, nrhs, lo, hi, order, mf):
    check(lib().cheby_filter(ctx.h, _ptr(out), _ptr(inp), nrhs, lo, hi, order, mf, _prec_of(inp),
                             _stream()), ctx.h)
    return out


def cheby_recursive_basis(ctx, phi, eta, lam_lo, lam_max, m, delta, nvec, mf):
    check(lib().cheby_recursive_basis(ctx.h, _ptr(phi), _ptr(eta), lam_lo, lam_max, m, delta, nvec,
                                      mf, _prec_of(eta), _stream()), ctx.h)
    return phi


def dwf_chiral_project(ctx, out, inp, sign, nrhs=1):
    check(lib().dwf_chiral_project(ctx.h, _ptr(out), _ptr(inp), sign, _prec_of(inp), nrhs,
                                   _stream()), ctx.h)
    return out


def block_orthonormalise(ctx, basis, nb, nplus, block):
    check(lib().block_orthonormalise(ctx.h, _ptr(basis), nb, nplus, _ivec(block), _stream()), ctx.h)
    return basis


class Coarse:
    """A dwf_coarse: the 9-point little Dirac operator of H_DW."""

    def __init__(self, handle, ctx, owned=True):
        self.h = handle
        self.ctx = ctx
        self.owned = owned
        dims = (C.c_int * 5)()
        check(lib().coarse_export(self.h, None, dims))
        self.Lc = tuple(dims[:4])
        self.nb = dims[4]
        self.nc = int(np.prod(self.Lc))

    def export(self):
        """FP64 operator as complex128 numpy (nc, 9, nb, nb)."""
        A = np.zeros((self.nc, 9, self.nb, self.nb), np.complex128)
        check(lib().coarse_export(self.h, _ptr(A), None))
        return A

    def close(self):
        if self.owned and self.h:
            lib().coarse_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def coarse_build(ctx, basis, nb, nplus, block, mf):
    h = C.c_void_p()
    check(lib().coarse_build(ctx.h, _ptr(basis), nb, nplus, _ivec(block), mf, _prec_of(basis),
                             C.byref(h), _stream()), ctx.h)
    return Coarse(h, ctx)


def coarse_apply(coarse, out, inp, nrhs=1, prec=F32):
    """prec F32 (CUDA cores) or TF32 (tcgen05 tensor cores, nb = 32, nrhs 16/32/64)."""
    check(lib().coarse_apply(coarse.h, _ptr(out), _ptr(inp), nrhs, prec, _stream()), coarse.ctx.h)
    return out


def coarse_apply_status(coarse):
    """Synchronise and raise if a bounded wait of an earlier tensor-core
    coarse_apply on this operator gave up."""
    check(lib().coarse_apply_status(coarse.h, _stream()), coarse.ctx.h)


def coarse_solve(coarse, e, r, tol, maxiter=1000):
    it = C.c_int()
    check(lib().coarse_solve(coarse.h, _ptr(e), _ptr(r), tol, maxiter, C.byref(it), _stream()),
          coarse.ctx.h)
    return it.value


def coarse_solve_multi(coarse, e, rhs, nrhs, tol, maxiter=1000, prec=F32):
    """CG on A^2 for nrhs right-hand sides at once ([nc][nb][nrhs] FP32);
    prec F32 (CUDA cores) or TF32 (tensor cores).  Returns the per-rhs
    iteration counts."""
    its = (C.c_int * nrhs)()
    check(lib().coarse_solve_multi(coarse.h, _ptr(e), _ptr(rhs), nrhs, tol, maxiter, its, prec, _stream()),
          coarse.ctx.h)
    return list(its)


def coarse_solve_rb(coarse, e, r, tol, maxiter=1000):
    """Red-black coarse solve (CG on the even Schur complement squared); returns
    the iteration count."""
    it = C.c_int()
    check(lib().coarse_solve_rb(coarse.h, _ptr(e), _ptr(r), tol, maxiter, C.byref(it), _stream()),
          coarse.ctx.h)
    return it.value


def coarse_deflate(coarse, v0, nev, nk, order, lam_lo, lam_max=0.0):
    """Chebyshev-preconditioned Lanczos deflation space of A^2 kept by the
    operator; returns the nev Ritz values (ascending).  nev = 0 drops it."""
    th = (C.c_double * max(nev, 1))()
    check(lib().coarse_deflate(coarse.h, _ptr(v0) if v0 is not None else None, nev, nk, order, lam_lo,
                               lam_max, th, _stream()), coarse.ctx.h)
    return [th[i] for i in range(nev)]


def coarse_export_deflation(coarse):
    """(V as complex128 numpy (nev, nc, nb), 1/theta) of the deflation space."""
    n = C.c_int()
    check(lib().coarse_export_deflation(coarse.h, None, None, C.byref(n)))
    V = np.zeros((n.value, coarse.nc, coarse.nb, 2), np.float32)
    ti = (C.c_double * max(n.value, 1))()
    check(lib().coarse_export_deflation(coarse.h, _ptr(V), ti, C.byref(n)))
    return V.astype(np.float64).view(np.complex128)[..., 0], np.array([ti[i] for i in range(n.value)])


def dwf_restrict(ctx, out, inp, basis, nb, block, nrhs=1):
    check(lib().dwf_restrict(ctx.h, _ptr(out), _ptr(inp), _ptr(basis), nb, _ivec(block), nrhs,
                             _prec_of(basis), _stream()), ctx.h)
    return out


def dwf_prolong(ctx, out, inp, basis, nb, block, nrhs=1, accumulate=0):
    check(lib().dwf_prolong(ctx.h, _ptr(out), _ptr(inp), _ptr(basis), nb, _ivec(block), nrhs,
                            _prec_of(basis), accumulate, _stream()), ctx.h)
    return out


def mg_params(block, nbasis, mf, *, subspace_mode=_lib.SUBSPACE_BATCH, lambda_lo=0.02,
              lambda_max=60.0, filter_order=60, delta=100, smooth=(0.5, 60.0, 12),
              coarse_tol=0.02, coarse_maxiter=500, nkrylov=8, maxiter=1000, graph=True,
              coarse_solver=_lib.COARSE_CG, deflation=(0, 0, 0, 0.0)):
    p = _lib.MGParams()
    p.block = (C.c_int * 4)(*block)
    p.nbasis, p.subspace_mode, p.mf = nbasis, subspace_mode, mf
    p.lambda_lo, p.lambda_max, p.filter_order, p.delta = lambda_lo, lambda_max, filter_order, delta
    p.smooth_lo, p.smooth_hi, p.smooth_order = smooth
    p.coarse_tol, p.coarse_maxiter, p.nkrylov, p.maxiter = coarse_tol, coarse_maxiter, nkrylov, maxiter
    p.no_graph = 0 if graph else 1
    p.coarse_solver = coarse_solver
    p.coarse_nev, p.coarse_lanczos, p.coarse_cheb_order, p.coarse_cheb_lo = deflation
    return p


class MG:
    """A dwf_mg: HDCR multigrid setup (basis + little Dirac operator)."""

    def __init__(self, ctx, params, eta):
        h = C.c_void_p()
        check(lib().mg_setup(ctx.h, C.byref(params), _ptr(eta), C.byref(h), _stream()), ctx.h)
        self.h = h
        self.ctx = ctx
        self.params = params
        self.coarse = Coarse(C.c_void_p(lib().mg_coarse(h)), ctx, owned=False)

    def basis(self):
        nb = self.params.nbasis
        out = torch.zeros(nb * 2 * self.ctx.half_numel(), dtype=torch.float32, device="cuda")
        check(lib().mg_export_basis(self.h, _ptr(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().mg_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mg_smooth(mg, out, inp):
    check(lib().mg_smooth(mg.h, _ptr(out), _ptr(inp), _stream()), mg.ctx.h)
    return out


def mg_precondition(mg, out, inp):
    check(lib().mg_precondition(mg.h, _ptr(out), _ptr(inp), _stream()), mg.ctx.h)
    return out


def set_f64_arithmetic(ctx, mode):
    """ARITH_FP64 (FP64 units) or ARITH_FLOAT_FLOAT (float-float on the FP32
    units) for the context's FP64-precision hopping launches."""
    check(lib().dwf_set_f64_arithmetic(ctx.h, int(mode)), ctx.h)


def hybrid_params(block, nbasis4, nbasis1, *, mass4=-0.95, filter4=(1.0, 60.0, 60),
                  filter1=(0.5, 60.0, 40), smooth1=(0.5, 60.0, 4), kcycle=2):
    """Parameters of the hybrid levels (Algorithm F): 4D blocks and basis size,
    the Wilson mass and filter (lo, hi, order) of the 4D subspace, the level-2
    basis size and its filter of H_1^2, the level-1 smoother (lo, hi, order;
    order 0, none, only with kcycle = 1) and the level-1 GCR iteration count."""
    h = _lib.HybridParams()
    h.block = (C.c_int * 4)(*block)
    h.nbasis4, h.mass4 = nbasis4, mass4
    h.lambda_lo4, h.lambda_max4, h.order4 = filter4
    h.nbasis1 = nbasis1
    h.lambda_lo1, h.lambda_max1, h.order1 = filter1
    h.smooth1_lo, h.smooth1_hi, h.smooth1_order = smooth1
    h.kcycle = kcycle
    return h


class HybridMG(MG):
    """A dwf_mg of the hybrid three-level multigrid (Algorithm F): eta4 holds
    nbasis4 FP64 4D fields as the slices of a full field with Ls = nbasis4,
    eta1 nbasis1 FP64 level-1 vectors ([nc1][nbasis4][Ls][nbasis1])."""

    def __init__(self, ctx, params, hparams, eta4, eta1):
        h = C.c_void_p()
        check(lib().mg_setup_hybrid(ctx.h, C.byref(params), C.byref(hparams), _ptr(eta4), _ptr(eta1), C.byref(h),
                                    _stream()), ctx.h)
        self.h = h
        self.ctx = ctx
        self.params = params
        self.hparams = hparams
        self.coarse = Coarse(C.c_void_p(lib().mg_coarse(h)), ctx, owned=False)
        L = ctx.L
        self.Lc = tuple(L[m] // hparams.block[m] for m in range(4))
        self.nc1 = int(np.prod(self.Lc))
        self.n1 = self.nc1 * hparams.nbasis4 * ctx.Ls

    def export(self, what):
        """0: the 4D basis (FP64); 1: B (FP64 [nc1][9][nb4][nb4]); 2: the level-2
        basis (FP32 [nc1][nb4][Ls][nb1]); 3: the level-2 stencil (FP64)."""
        hp = self.hparams
        n = {0: 2 * self.ctx.Vh * 12 * hp.nbasis4,
             1: self.nc1 * 9 * hp.nbasis4 ** 2, 2: self.n1 * hp.nbasis1, 3: self.nc1 * 9 * hp.nbasis1 ** 2}[what]
        dt = torch.float32 if what == 2 else torch.float64
        out = torch.zeros(2 * n, dtype=dt, device="cuda")
        check(lib().mg_hybrid_export(self.h, what, _ptr(out)), self.ctx.h)
        return out

    def level1(self, op, out, inp, nvec=1):
        """0: M_1, 1: H_1, 2: P1^dag, 3: P1, 4: P2^dag, 5: P2, 6: the level-1 W-cycle solve."""
        check(lib().mg_hybrid_level1(self.h, op, _ptr(out), _ptr(inp), nvec, _stream()), self.ctx.h)
        return out


def mg_solve(mg, x, b, tol):
    st = SolveStats()
    check(lib().mg_solve(mg.h, _ptr(x), _ptr(b), tol, C.byref(st), _stream()), mg.ctx.h)
    return st.as_dict()


def dwf_force(ctx, force, X, masses):
    """force (complex128 device tensor, gauge layout) += sum_i G_i for the even
    solutions X (npf half fields back to back, FP64 or FP32)."""
    m = (C.c_double * len(masses))(*masses)
    check(lib().dwf_force(ctx.h, _ptr(force), _ptr(X), m, len(masses), _prec_of(X), _stream()), ctx.h)
    return force


def dwf_ratio_force(ctx, force, X, phi, m1, m2):
    """force += sum_i G_r,i of the Hasenbusch ratio factors phi_i^dag M2 (M1^dag
    M1)^-1 M2^dag phi_i (X_i = (M1^dag M1)^-1 M2^dag phi_i; X and phi hold the
    factors' even half fields back to back, same precision)."""
    n = len(m1)
    a = (C.c_double * n)(*[float(m) for m in m1])
    b = (C.c_double * n)(*[float(m) for m in m2])
    check(lib().dwf_ratio_force(ctx.h, _ptr(force), _ptr(X), _ptr(phi), a, b, n, _prec_of(X), _stream()),
          ctx.h)
    return force


def dwf_pf_action(ctx, phi, X, masses):
    """sum_i 2 Re <phi_i, X_i> - |M_pc(m_i) X_i|^2 (FP64 even half fields back to back)."""
    n = len(masses)
    m = (C.c_double * n)(*[float(v) for v in masses])
    S = C.c_double()
    check(lib().dwf_pf_action(ctx.h, C.byref(S), _ptr(phi), _ptr(X), m, n, _stream()), ctx.h)
    return S.value


def rbcg_normal_solve(ctx, x, phi, mf, tol, maxiter=100000, policy=_lib.SOLVE_MIXED_F32):
    """x = (M_pc^dag M_pc)^-1 phi on the even parity (FP64 device half fields)."""
    st = SolveStats()
    check(lib().rbcg_normal_solve(ctx.h, _ptr(x), _ptr(phi), mf, tol, maxiter, policy, C.byref(st),
                                  _stream()), ctx.h)
    return st.as_dict()


def cgnr_solve(ctx, x, b, mf, tol, maxiter=100000):
    """Unpreconditioned FP64 CGNR on the full lattice (full FP64 device
    fields).  Returns the solver statistics as a dict."""
    st = SolveStats()
    check(lib().cgnr_solve(ctx.h, _ptr(x), _ptr(b), mf, tol, maxiter, C.byref(st), _stream()), ctx.h)
    return st.as_dict()


def _batch_solve(fn, ctx, x, b, masses, tol, maxiter, policy):
    n = len(masses)
    mf = (C.c_double * n)(*[float(m) for m in masses])
    st = (SolveStats * n)()
    check(fn(ctx.h, _ptr(x), _ptr(b), mf, n, tol, maxiter, policy, st, _stream()), ctx.h)
    return [s.as_dict() for s in st]


def rbcg_solve_batch(ctx, x, b, masses, tol, maxiter=100000, policy=_lib.SOLVE_MIXED_F32):
    """Red-black CGNR for len(masses) full FP64 fields stored back to back in
    b (host or device; x the same kind), rhs i with mass masses[i], solved as
    one batch.  Returns one stats dict per rhs."""
    return _batch_solve(lib().rbcg_solve_batch, ctx, x, b, masses, tol, maxiter, policy)


def rbcg_normal_solve_batch(ctx, x, phi, masses, tol, maxiter=100000, policy=_lib.SOLVE_MIXED_F32):
    """x_i = (M_pc(m_i)^dag M_pc(m_i))^-1 phi_i for FP64 even half fields
    stored back to back on the device.  Returns one stats dict per rhs."""
    return _batch_solve(lib().rbcg_normal_solve_batch, ctx, x, phi, masses, tol, maxiter, policy)


def dwf_measure_fma_peaks():
    """(FP64, FP32) FMA rates of this GPU in TFLOP/s, measured by the library."""
    a, b = C.c_double(), C.c_double()
    check(lib().dwf_measure_fma_peaks(C.byref(a), C.byref(b), _stream()))
    return a.value, b.value


def dwf_autotune(ctx, prec=F32, reps=20):
    """Pick the fastest hopping-kernel variant for this lattice; returns
    (variant, ms per launch)."""
    ms = C.c_double()
    check(lib().dwf_autotune(ctx.h, prec, reps, C.byref(ms), _stream()), ctx.h)
    return lib().dwf_get_hop_variant(ctx.h, prec), ms.value


def dwf_set_hop_variant(ctx, prec, variant):
    check(lib().dwf_set_hop_variant(ctx.h, prec, variant), ctx.h)
