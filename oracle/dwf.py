"""Shamir domain wall fermion operators in FP64 (oracle; test infrastructure only).

Paper: Boyle & Yamaguchi, arXiv:2103.05034, Section 2.
  Eq. (1)  D_W(M) = M + 4 - 1/2 D_hop
  Eq. (2)  D_hop = (1 - gamma_mu) U_mu(x) delta_{x+mu,y} + (1 + gamma_mu) U_mu^dag(y) delta_{x-mu,y}
  Eq. (4)  D_DW: D_par on the diagonal of the Ls x Ls fifth-dimension matrix,
           -P_- above it, -P_+ below it, m P_+ in the top-right corner and
           m P_- in the bottom-left corner
  Eq. (5)  D_par = 5 - M5 - 1/2 D_hop
  Eq. (6)  H_DW = Gamma_5 D_DW,  Gamma_5 = gamma_5 R_5 (R_5: s -> Ls-1-s)
  Sec. 5.1 red-black (even-odd) Schur form M_ee - M_eo M_oo^-1 M_oe

Everything is written on full-lattice arrays with full 4x4 spin matrices and
np.roll for the neighbours: no spin projection, no checkerboarded storage.
A "half" (single-parity) field is a full-lattice array that is zero on the
other parity.  The sum over mu in Eq. (2) is implied; U_mu^dag(y) with
y = x - mu is the link U_mu(x - mu) daggered.  Boundaries are periodic.

Readings of the paper taken here (the paper does not fix them):
  * gamma basis: the chiral basis gamma_k = [[0, -i s_k], [i s_k, 0]],
    gamma_4 = [[0, 1], [1, 0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4
    = diag(1, 1, -1, -1); P_+- = (1 +- gamma_5)/2.
  * M5 = 1.8 (the workloads' value).
"""
from __future__ import annotations

import numpy as np

# ---------------------------------------------------------------- gamma matrices
_sig = [np.array([[0, 1], [1, 0]], complex),
        np.array([[0, -1j], [1j, 0]], complex),
        np.array([[1, 0], [0, -1]], complex)]
_Z2 = np.zeros((2, 2), complex)
_I2 = np.eye(2, dtype=complex)


def _chiral_gamma(k):
    if k < 3:
        return np.block([[_Z2, -1j * _sig[k]], [1j * _sig[k], _Z2]])
    return np.block([[_Z2, _I2], [_I2, _Z2]])


GAMMA = np.array([_chiral_gamma(k) for k in range(4)])  # gamma_1..gamma_4 (x,y,z,t)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=complex)
P_PLUS = 0.5 * (ID4 + GAMMA5)
P_MINUS = 0.5 * (ID4 - GAMMA5)

_AX = (3, 2, 1, 0)  # array axis of direction mu in a (T, Z, Y, X, ...) array


def shift(f, mu, sign):
    """The field f(x + sign*mu) at site x (periodic boundaries)."""
    return np.roll(f, -sign, axis=_AX[mu])


def dagger(U):
    return np.conj(np.swapaxes(U, -1, -2))


# ---------------------------------------------------------------- parity
def parity_mask(L):
    """1.0 on even sites (x+y+z+t even), 0.0 on odd sites; shape (T,Z,Y,X)."""
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                             np.arange(Lx), indexing="ij")
    return ((x + y + z + t) % 2 == 0).astype(float)


def project_parity(psi, L, parity):
    """Keep the sites of one parity (0 even, 1 odd), zero the rest."""
    m = parity_mask(L)
    if parity == 1:
        m = 1.0 - m
    return psi * m.reshape(m.shape + (1,) * (psi.ndim - 4))


def lattice_dims(psi):
    T, Z, Y, X = psi.shape[:4]
    return (X, Y, Z, T)


# ---------------------------------------------------------------- Eq. (2)
def apply_spin(G, psi):
    """Apply a 4x4 spin matrix to a (..., 4, 3) spinor field."""
    return np.einsum("ij,...jc->...ic", G, psi)


def apply_color(U4, psi):
    """Apply a per-4D-site colour matrix (T,Z,Y,X,3,3) to a (T,Z,Y,X,Ls,4,3) field."""
    return np.einsum("tzyxab,tzyxsib->tzyxsia", U4, psi)


def dhop(U, psi, dag=False):
    """D_hop psi, Eq. (2), or its adjoint when dag=True.

    The adjoint follows from transposing Eq. (2): the forward term becomes
    (1 + gamma_mu) U_mu(x) psi(x+mu) and the backward term
    (1 - gamma_mu) U_mu^dag(x-mu) psi(x-mu).
    """
    out = np.zeros_like(psi)
    sgn = -1.0 if dag else 1.0
    for mu in range(4):
        Umu = U[..., mu, :, :]
        fwd = apply_color(Umu, shift(psi, mu, +1))
        out += apply_spin(ID4 - sgn * GAMMA[mu], fwd)
        bwd = apply_color(dagger(shift(Umu, mu, -1)), shift(psi, mu, -1))
        out += apply_spin(ID4 + sgn * GAMMA[mu], bwd)
    return out


def dhop_direction(U, psi, mu, sign, dag=False):
    """One of the eight terms of Eq. (2): sign=+1 the hop from x+mu, -1 from x-mu."""
    s = -1.0 if dag else 1.0
    Umu = U[..., mu, :, :]
    if sign > 0:
        return apply_spin(ID4 - s * GAMMA[mu], apply_color(Umu, shift(psi, mu, +1)))
    return apply_spin(ID4 + s * GAMMA[mu],
                      apply_color(dagger(shift(Umu, mu, -1)), shift(psi, mu, -1)))


# ---------------------------------------------------------------- Eq. (4) fifth dimension
def fifth_dim_matrix(Ls, M5, mf):
    """The site-local part of D_DW, Eq. (4) without the -1/2 D_hop of Eq. (5):
    K[s, s'] (an Ls x Ls array of 4x4 spin matrices)."""
    K = np.zeros((Ls, Ls, 4, 4), dtype=complex)
    for s in range(Ls):
        K[s, s] = (5.0 - M5) * ID4
        if s + 1 < Ls:
            K[s, s + 1] = -P_MINUS
        if s - 1 >= 0:
            K[s, s - 1] = -P_PLUS
    K[0, Ls - 1] += mf * P_PLUS
    K[Ls - 1, 0] += mf * P_MINUS
    return K


def apply_fifth(K, psi):
    """(K psi)_s = sum_s' K[s,s'] psi_s' at every 4D site."""
    return np.einsum("abij,tzyxbjc->tzyxaic", K, psi)


def k_dense(K):
    """K as a (4 Ls) x (4 Ls) matrix, index (s, spin)."""
    Ls = K.shape[0]
    return K.transpose(0, 2, 1, 3).reshape(4 * Ls, 4 * Ls)


def apply_dense_sitelocal(Kd, psi):
    Ls = psi.shape[4]
    v = psi.reshape(psi.shape[:4] + (4 * Ls, 3))
    return np.einsum("ab,tzyxbc->tzyxac", Kd, v).reshape(psi.shape)


def ddw(U, psi, M5, mf, dag=False):
    """D_DW psi, Eq. (4) with Eq. (5); dag=True gives D_DW^dag."""
    Ls = psi.shape[4]
    Kd = k_dense(fifth_dim_matrix(Ls, M5, mf))
    if dag:
        Kd = Kd.conj().T
    return apply_dense_sitelocal(Kd, psi) - 0.5 * dhop(U, psi, dag=dag)


def gamma5_r5(psi):
    """Gamma_5 psi = gamma_5 R_5 psi: (Gamma_5 psi)_s = gamma_5 psi_{Ls-1-s}."""
    return apply_spin(GAMMA5, psi[:, :, :, :, ::-1])


def hdw(U, psi, M5, mf):
    """H_DW psi = Gamma_5 D_DW psi, Eq. (6)."""
    return gamma5_r5(ddw(U, psi, M5, mf))


def mdagm(U, psi, M5, mf):
    """D_DW^dag D_DW psi (equal to H_DW^2 psi)."""
    return ddw(U, ddw(U, psi, M5, mf), M5, mf, dag=True)


# ---------------------------------------------------------------- red-black Schur form
def mooee(psi, M5, mf, dag=False):
    """M_ee (or M_oo): the site-local fifth-dimension part of D_DW."""
    Kd = k_dense(fifth_dim_matrix(psi.shape[4], M5, mf))
    if dag:
        Kd = Kd.conj().T
    return apply_dense_sitelocal(Kd, psi)


def mooee_inv(psi, M5, mf, dag=False):
    """M_ee^-1 psi by dense solve of the (4 Ls) x (4 Ls) site-local matrix."""
    Kd = k_dense(fifth_dim_matrix(psi.shape[4], M5, mf))
    if dag:
        Kd = Kd.conj().T
    return apply_dense_sitelocal(np.linalg.inv(Kd), psi)


def meo(U, psi, out_parity, dag=False):
    """M_eo (out_parity 0) or M_oe (out_parity 1): -1/2 D_hop between parities.
    psi must vanish on the out_parity sites."""
    L = lattice_dims(psi)
    return project_parity(-0.5 * dhop(U, psi, dag=dag), L, out_parity)


def mpc(U, psi_e, M5, mf):
    """M_pc psi_e = (M_ee - M_eo M_oo^-1 M_oe) psi_e (the Schur form used for the
    red-black CGNR baseline, Table 5 row 'prec-CGNR (M_ee - M_eo M_oo^-1 M_oe)')."""
    t = mooee_inv(meo(U, psi_e, 1), M5, mf)
    return mooee(psi_e, M5, mf) - meo(U, t, 0)


def mpc_dag(U, psi_e, M5, mf):
    """M_pc^dag psi_e = (M_ee^dag - M_oe^dag M_oo^-dag M_eo^dag) psi_e."""
    t = mooee_inv(meo(U, psi_e, 1, dag=True), M5, mf, dag=True)
    return mooee(psi_e, M5, mf, dag=True) - meo(U, t, 0, dag=True)


def mpcdag_mpc(U, psi_e, M5, mf):
    return mpc_dag(U, mpc(U, psi_e, M5, mf), M5, mf)


def mpc2(U, psi_e, M5, mf):
    """The second Schur form of Table 5, (1 - M_ee^-1 M_eo M_oo^-1 M_oe) psi_e,
    which is M_ee^-1 M_pc psi_e."""
    return mooee_inv(mpc(U, psi_e, M5, mf), M5, mf)


def mpc2_dag(U, psi_e, M5, mf):
    """(1 - M_ee^-1 M_eo M_oo^-1 M_oe)^dag psi_e = M_pc^dag M_ee^-dag psi_e."""
    return mpc_dag(U, mooee_inv(psi_e, M5, mf, dag=True), M5, mf)


# ---------------------------------------------------------------- inner products
def inner(a, b):
    """<a, b> = sum conj(a) b."""
    return np.vdot(a.ravel(), b.ravel())


def norm2(a):
    return float(np.vdot(a.ravel(), a.ravel()).real)
