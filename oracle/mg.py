"""HDCR multigrid: V(1,1) preconditioner and flexible GCR in FP64 (oracle;
test infrastructure only).

Paper: arXiv:2103.05034.
  Sec. 3.1, Eq. (19): Q = P A^-1 P^dag (the subspace inverse)
  Sec. 3.3, Eqs. (26)-(28): x1 = x0 + S r0, x2 = x1 + Q r1, x3 = x2 + S r2,
           used as a preconditioner on the current residual (x0 = 0)
  Sec. 4, Table 1 (Algorithms A, B): outer pGCR(H_DW), smoother
           S_cheb([0.5, 60], 12), coarsening of H_DW, coarse CGNR to a
           relative tolerance of 0.02
  Sec. 2.1: a Gamma_5-hermitian system is solved as H_DW x = Gamma_5 b

Readings:
  * pGCR is flexible (variable-preconditioner) GCR restarted every nkrylov
    directions, with the true residual recomputed at each restart.
  * The smoother for H_DW takes M = M^dag = H_DW, so M^dag M = H_DW^2.
  * The coarse solve is CG on A^2 e = A r_c to relative residual coarse_tol.
  * Convergence is judged on ||Gamma_5 b - H x|| = ||b - D_DW x||.
"""
from __future__ import annotations

import numpy as np

from . import cheby, coarse, dwf


class MGCounter:
    def __init__(self):
        self.fine = 0
        self.coarse = 0


def vcycle(apply_H, r0, basis, A, block, smooth, coarse_tol, coarse_maxiter, cnt):
    """The V(1,1) correction for residual r0 (x0 = 0), Eqs. (26)-(28)."""
    a, b, N = smooth
    x1, n = cheby.smoother_apply(apply_H, apply_H, r0, a, b, N)
    cnt.fine += n
    r1 = r0 - apply_H(x1)
    cnt.fine += 1
    rc = coarse.restrict(basis, r1, block)
    ec, it = coarse.coarse_cgnr(A, rc, coarse_tol, coarse_maxiter)
    cnt.coarse += it
    x2 = x1 + coarse.prolong(basis, ec, block)
    r2 = r0 - apply_H(x2)
    cnt.fine += 1
    s2, n = cheby.smoother_apply(apply_H, apply_H, r2, a, b, N)
    cnt.fine += n
    return x2 + s2


def pgcr(apply_H, rhs, precond, tol, maxiter, nkrylov, cnt):
    """Flexible GCR on H x = rhs; stops when ||rhs - H x|| <= tol ||rhs||.
    Returns (x, outer iterations, residual history)."""
    x = np.zeros_like(rhs)
    r = rhs.copy()
    bnorm = np.sqrt(dwf.norm2(rhs))
    hist = [1.0]
    it = 0
    while it < maxiter:
        zs, ws = [], []
        for _ in range(nkrylov):
            z = precond(r)
            w = apply_H(z)
            cnt.fine += 1
            for zj, wj in zip(zs, ws):
                beta = dwf.inner(wj, w) / dwf.norm2(wj)
                w = w - beta * wj
                z = z - beta * zj
            alpha = dwf.inner(w, r) / dwf.norm2(w)
            x = x + alpha * z
            r = r - alpha * w
            zs.append(z)
            ws.append(w)
            it += 1
            res = np.sqrt(dwf.norm2(r)) / bnorm
            hist.append(res)
            if res <= tol or it >= maxiter:
                break
        r = rhs - apply_H(x)
        cnt.fine += 1
        if np.sqrt(dwf.norm2(r)) / bnorm <= tol:
            break
    return x, it, hist


def mg_solve(U, b, basis, A, block, M5, mf, tol, smooth=(0.5, 60.0, 12),
             coarse_tol=0.02, coarse_maxiter=500, maxiter=200, nkrylov=8):
    """HDCR solve of D_DW x = b with outer pGCR(H_DW) and the V(1,1) preconditioner."""
    apply_H = lambda v: dwf.hdw(U, v, M5, mf)
    cnt = MGCounter()
    pre = lambda r: vcycle(apply_H, r, basis, A, block, smooth, coarse_tol, coarse_maxiter, cnt)
    x, it, hist = pgcr(apply_H, dwf.gamma5_r5(b), pre, tol, maxiter, nkrylov, cnt)
    return x, it, hist, cnt
