"""Pseudofermion action and its gauge-link derivative in FP64 (oracle; test
infrastructure only).

The paper places its solvers inside Hybrid Monte Carlo (Sec. 6: solves per
molecular-dynamics step, Hasenbusch factors) but prints no force formula; this
is derived from first principles for the red-black operator of Sec. 5.1.

  S(U) = sum_i phi_i^dag (M_i^dag M_i)^-1 phi_i,  M_i = M_pc(m_i) (even sites)
  X = (M^dag M)^-1 phi,  Y = M X
  dS = -2 Re Y^dag dM X,  dM = -dM_eo M_oo^-1 M_oe - M_eo M_oo^-1 dM_oe
  With X_o = M_oo^-1 M_oe X and Y_o = M_oo^-dag M_eo^dag Y, and the full
  fields X' = X + X_o, Y' = Y + Y_o:  dS = -Re Y'^dag dD_hop X'.
  For U_mu(x) -> exp(eps Q) U_mu(x), Q in su(3):
    dS/deps = -Re sum tr(Q Z),  Z_mu(x) = U_mu(x) A_mu(x) - B_mu(x) U_mu(x)^dag
    A_mu(x)_{ab} = sum_{s,i,j} (1 - gamma_mu)_{ij} X'_{s j a}(x+mu) conj(Y'_{s i b}(x))
    B_mu(x)_{ab} = sum_{s,i,j} (1 + gamma_mu)_{ij} X'_{s j a}(x) conj(Y'_{s i b}(x+mu))
  The force G = TA(Z) (TA(M) = (M - M^dag)/2 - tr(M - M^dag)/6) then gives
  dS/deps = sum Re tr(G^dag Q) for every traceless anti-hermitian Q.

Hasenbusch ratio factor (the intermediate determinant ratios of Sec. 6,
det[M(m1)^dag M(m1)] / det[M(m2)^dag M(m2)]), represented by
  S_r(U) = phi^dag M2 (M1^dag M1)^-1 M2^dag phi,  M_i = M_pc(m_i):
  chi = M2^dag phi,  X = (M1^dag M1)^-1 chi,  Y = M1 X,
  dS_r = 2 Re phi^dag dM2 X - 2 Re Y^dag dM1 X.
  Each term is a bilinear -2 Re L^dag dM R of the form above with its full
  fields R' = R + M_oo^-1 M_oe R, L' = L + M_oo^-dag M_eo^dag L (at that
  term's mass), so G_r = G(X'_1, Y'_1) - G(X'_2, phi'_2).  With m1 = m2 the
  action is phi^dag phi, independent of U, and G_r vanishes.
"""
from __future__ import annotations

import numpy as np

from . import dwf, krylov


def traceless_antihermitian(M):
    A = 0.5 * (M - dwf.dagger(M))
    tr = np.trace(A, axis1=-2, axis2=-1)
    return A - (tr / 3.0)[..., None, None] * np.eye(3)


def solve_normal(U, phi, M5, mf, tol=1e-13):
    X, _, _ = krylov.cg(lambda v: dwf.mpcdag_mpc(U, v, M5, mf), phi, tol, 100000)
    return X


def action(U, phis, masses, M5, tol=1e-13):
    """S = sum_i phi_i^dag (M^dag M)^-1 phi_i by the estimator
    2 Re <phi, X> - <X, M^dag M X>, whose error is quadratic in the solve error."""
    S = 0.0
    for phi, mf in zip(phis, masses):
        X = solve_normal(U, phi, M5, mf, tol)
        S += 2 * dwf.inner(phi, X).real - dwf.inner(X, dwf.mpcdag_mpc(U, X, M5, mf)).real
    return S


def force_fields(U, phi, M5, mf, tol=1e-13):
    """The full fields X', Y' of the derivation above."""
    X = solve_normal(U, phi, M5, mf, tol)
    Y = dwf.mpc(U, X, M5, mf)
    Xo = dwf.mooee_inv(dwf.meo(U, X, 1), M5, mf)
    Yo = dwf.mooee_inv(dwf.meo(U, Y, 1, dag=True), M5, mf, dag=True)
    return X + Xo, Y + Yo


def bilinear_fields(U, R, L, M5, mf):
    """Full fields R', L' of a bilinear -2 Re L^dag dM_pc R (R, L even)."""
    Ro = dwf.mooee_inv(dwf.meo(U, R, 1), M5, mf)
    Lo = dwf.mooee_inv(dwf.meo(U, L, 1, dag=True), M5, mf, dag=True)
    return R + Ro, L + Lo


def force_from_fields(U, Xf, Yf):
    """G_mu(x) = TA(U A - B U^dag) for the fields X', Y'.  (T,Z,Y,X,4,3,3)."""
    G = np.zeros_like(U)
    for mu in range(4):
        Xp = dwf.shift(Xf, mu, +1)
        Yp = dwf.shift(Yf, mu, +1)
        Pm = dwf.ID4 - dwf.GAMMA[mu]
        Pp = dwf.ID4 + dwf.GAMMA[mu]
        Amu = np.einsum("ij,tzyxsja,tzyxsib->tzyxab", Pm, Xp, Yf.conj())
        Bmu = np.einsum("ij,tzyxsja,tzyxsib->tzyxab", Pp, Xf, Yp.conj())
        Umu = U[..., mu, :, :]
        G[..., mu, :, :] = traceless_antihermitian(Umu @ Amu - Bmu @ dwf.dagger(Umu))
    return G


def force(U, phis, masses, M5, tol=1e-13):
    G = np.zeros_like(U)
    for phi, mf in zip(phis, masses):
        Xf, Yf = force_fields(U, phi, M5, mf, tol)
        G += force_from_fields(U, Xf, Yf)
    return G


def ratio_action(U, phi, m1, m2, M5, tol=1e-13):
    """S_r = phi^dag M2 (M1^dag M1)^-1 M2^dag phi by the estimator
    2 Re <chi, X> - <X, M1^dag M1 X> (chi = M2^dag phi)."""
    chi = dwf.mpc_dag(U, phi, M5, m2)
    X = solve_normal(U, chi, M5, m1, tol)
    return 2 * dwf.inner(chi, X).real - dwf.inner(X, dwf.mpcdag_mpc(U, X, M5, m1)).real


def ratio_force(U, phi, m1, m2, M5, tol=1e-13):
    """G_r of the ratio factor (derivation in the module docstring)."""
    chi = dwf.mpc_dag(U, phi, M5, m2)
    X = solve_normal(U, chi, M5, m1, tol)
    Y = dwf.mpc(U, X, M5, m1)
    Xf1, Yf1 = bilinear_fields(U, X, Y, M5, m1)
    Xf2, Pf2 = bilinear_fields(U, X, phi, M5, m2)
    return force_from_fields(U, Xf1, Yf1) - force_from_fields(U, Xf2, Pf2)


def exp_su3(Q):
    """exp(Q) for anti-hermitian Q via the eigendecomposition of the hermitian -iQ."""
    w, V = np.linalg.eigh(-1j * Q)
    return np.einsum("...ij,...j,...kj->...ik", V, np.exp(1j * w), V.conj())


def finite_difference(U, phis, masses, M5, Q, eps, tol=1e-13):
    """Central difference (S(e^{eps Q} U) - S(e^{-eps Q} U)) / (2 eps)."""
    Up = np.einsum("...ij,...jk->...ik", exp_su3(eps * Q), U)
    Um = np.einsum("...ij,...jk->...ik", exp_su3(-eps * Q), U)
    return (action(Up, phis, masses, M5, tol) - action(Um, phis, masses, M5, tol)) / (2 * eps)
