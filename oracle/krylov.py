"""Krylov solvers and the power method in FP64 (oracle; test infrastructure only).

Paper: arXiv:2103.05034.
  Sec. 2.1, Eq. (9): CG on the normal equations M_pc^dag M_pc psi = eta
  Sec. 5.1, Table 5: red-black preconditioned CGNR with the Schur complement
           M_ee - M_eo M_oo^-1 M_oe (the baseline the multigrid must beat)
  Sec. 3.4: the power method gives lambda_max of M^dag M

Readings (the paper gives no details of these standard algorithms):
  * CG is textbook Hestenes-Stiefel CG.
  * The red-black solve prepares the even source b'_e = b_e - M_eo M_oo^-1 b_o,
    solves M_pc^dag M_pc x_e = M_pc^dag b'_e, and reconstructs
    x_o = M_oo^-1 (b_o - M_oe x_e).  The second Schur form of Table 5 solves
    M2 x_e = M_ee^-1 b'_e with M2 = M_ee^-1 M_pc by CG on its normal equations.
  * A solve is judged by the true relative residual ||b - D_DW x|| / ||b||.
"""
from __future__ import annotations

import numpy as np

from . import dwf


def cg(apply_A, b, tol, maxiter, x0=None):
    """Conjugate gradients on a hermitian positive definite operator.
    Stops when ||b - A x|| <= tol ||b|| (the recursively updated residual).
    Returns (x, iterations, residual history)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = dwf.norm2(r)
    bb = dwf.norm2(b)
    hist = [np.sqrt(rr / bb)]
    k = 0
    while k < maxiter and rr > tol * tol * bb:
        Ap = apply_A(p)
        alpha = rr / dwf.inner(p, Ap).real
        x += alpha * p
        r -= alpha * Ap
        rr_new = dwf.norm2(r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        k += 1
        hist.append(np.sqrt(rr / bb))
    return x, k, hist


def rb_prepare_source(U, b, M5, mf):
    """Even-parity right-hand side M_pc^dag (b_e - M_eo M_oo^-1 b_o)."""
    L = dwf.lattice_dims(b)
    be = dwf.project_parity(b, L, 0)
    bo = dwf.project_parity(b, L, 1)
    bprime = be - dwf.meo(U, dwf.mooee_inv(bo, M5, mf), 0)
    return dwf.mpc_dag(U, bprime, M5, mf)


def rb_reconstruct(U, b, xe, M5, mf):
    """Full solution from the even part: x_o = M_oo^-1 (b_o - M_oe x_e)."""
    L = dwf.lattice_dims(b)
    bo = dwf.project_parity(b, L, 1)
    xo = dwf.mooee_inv(bo - dwf.meo(U, xe, 1), M5, mf)
    return xe + xo


def rbcg_solve(U, b, M5, mf, tol, maxiter=100000):
    """Red-black CGNR solve of D_DW x = b.  tol applies to the CG residual of
    the even normal equations; the caller judges the true residual."""
    rhs = rb_prepare_source(U, b, M5, mf)
    xe, it, hist = cg(lambda v: dwf.mpcdag_mpc(U, v, M5, mf), rhs, tol, maxiter)
    return rb_reconstruct(U, b, xe, M5, mf), it, hist


def rbcg2_solve(U, b, M5, mf, tol, maxiter=100000):
    """Red-black CGNR with the second Schur form of Table 5: CG on
    M2^dag M2 x_e = M2^dag M_ee^-1 b'_e, M2 = 1 - M_ee^-1 M_eo M_oo^-1 M_oe
    (b'_e = b_e - M_eo M_oo^-1 b_o, x_o reconstructed as for the first form)."""
    L = dwf.lattice_dims(b)
    be = dwf.project_parity(b, L, 0)
    bo = dwf.project_parity(b, L, 1)
    bprime = be - dwf.meo(U, dwf.mooee_inv(bo, M5, mf), 0)
    rhs = dwf.mpc2_dag(U, dwf.mooee_inv(bprime, M5, mf), M5, mf)
    xe, it, hist = cg(lambda v: dwf.mpc2_dag(U, dwf.mpc2(U, v, M5, mf), M5, mf), rhs, tol, maxiter)
    return rb_reconstruct(U, b, xe, M5, mf), it, hist


def true_residual(U, x, b, M5, mf):
    """||b - D_DW x|| / ||b||."""
    return np.sqrt(dwf.norm2(b - dwf.ddw(U, x, M5, mf)) / dwf.norm2(b))


def power_max(apply_A, v0, iters):
    """Power method estimate of the largest eigenvalue of a hermitian positive
    operator: v <- A v / ||A v||, lambda = <v, A v>."""
    v = v0 / np.sqrt(dwf.norm2(v0))
    lam = 0.0
    for _ in range(iters):
        w = apply_A(v)
        lam = dwf.inner(v, w).real
        v = w / np.sqrt(dwf.norm2(w))
    return lam
