"""Hybrid-M^dag M multigrid (Algorithm F) in FP64 (oracle; test infrastructure
only).

Paper: arXiv:2103.05034.
  Eq. (1): D_W(M) = M + 4 - 1/2 D_hop (the four dimensional Wilson operator)
  Sec. 3.1, Eqs. (14), (18): block basis, restrictor P^dag and prolongator P,
           little Dirac operator A = P^dag M P (nearest neighbour)
  Sec. 3.4 (end): for a four dimensional D_W coarsening the vectors are
           projected with (1 +- gamma_5)/2, for the five dimensional one with
           (1 +- Gamma_5)/2; the sign relation makes gamma_5 (Gamma_5) exact
           on the coarse space
  Sec. 4, Algorithms E and F and the table of Algorithm F: the first
           coarsening represents D_W on 4D blocks (2^4 x 1) with a basis from a
           Chebyshev filter of D_W^dag D_W at a near-critical Wilson mass, and
           the coarse space keeps the fifth dimension (a coarse domain wall
           operator built from the coarse D_W); a second coarsening of H_DW on
           that space with blocks spanning the coarse fifth dimension
           (1^4 x Ls) gives a four dimensional coarse-coarse grid, solved by
           deflated CGNR; a fixed-iteration W-cycle makes two coarse-coarse
           corrections for every coarse grid step
  Sec. 4, table of fine-matrix counts for Algorithms F and G: two solves in
           the doubly coarsened space per outer iteration

Readings (the paper does not spell these out):
  * Level 1 is P1^dag D_DW P1 with P1 the 4D block basis applied on every
    s-slice.  Each 4D basis vector has a definite chirality chi_k, so
    P1^dag P_+- P1 is the sign pattern of the basis index and level 1 is a
    coarse Shamir operator: M_1 = K_chi (x) 1 + B (x) 1_s, where K_chi is the
    Ls x Ls scalar fifth-dimension matrix of Eq. (4) for chirality chi and
    B = P4^dag (-1/2 D_hop) P4 is a 9-point stencil of nb4 x nb4 blocks.
  * 4D subspace: nb4 Gaussian 4D fields, each filtered by
    T_order(x(D_W(m)^dag D_W(m))) on [lo, hi] (the batch form of Sec. 3.4),
    the first half projected with (1 + gamma_5)/2 and the rest with
    (1 - gamma_5)/2, then block orthonormalised (MGS twice per block and
    chirality).  The paper's Wilson mass -0.95 and its recursive filter are
    parameters of the same construction.
  * Level 2 coarsens H_1 = Gamma5_1 M_1, Gamma5_1 = chi_k R_5 (the sign of the
    basis index and s -> Ls-1-s), on blocks of one level-1 site spanning all
    s; basis: nb2 Gaussian level-1 vectors filtered by T_order(x(H_1^2)),
    (1 +- Gamma5_1)/2 halves, orthonormalised per site.
  * Fine level: flexible GCR on H_DW x = Gamma_5 b with the V(1,1)
    preconditioner of Sec. 3.3 (smoother on H_DW); this is pGCR(M) of the
    table with Gamma_5 moved into the preconditioner (same residual norms).
    Its coarse correction is P1 e with e an approximate solution of
    H_1 e = P1^dag r.
  * Level-1 solve: kcycle (2) iterations of flexible GCR on H_1 from zero
    with no tolerance test, each preconditioned by a level-1 V(1,1): a
    Chebyshev smoother on H_1 around the coarse-coarse correction
    P2 A_2^-1 P2^dag, A_2^-1 by CG on A_2^2 to the coarse tolerance.  So
    every fine outer iteration makes kcycle coarse-coarse solves.  The
    smoother may be left out (order 0) only with kcycle = 1: without it the
    preconditioner K = P2 A_2^-1 P2^dag satisfies K H_1 K = K, and a second
    GCR direction would vanish.

Layouts: 4D fields (T,Z,Y,X,4,3); level-1 fields (Tc,Zc,Yc,Xc, nb4, Ls)
(basis index, then s); level-2 vectors (Tc,Zc,Yc,Xc, nb2).
"""
from __future__ import annotations

import numpy as np

from . import cheby, coarse, dwf, mg

SITE = (1, 1, 1, 1)  # level-2 blocks: one level-1 site (and all of its s)


# ---------------------------------------------------------------- Eq. (1) in 4D
def wilson(U, psi, mass, dag=False):
    """D_W(mass) psi = (mass + 4) psi - 1/2 D_hop psi on a 4D field (Eq. 1);
    dag=True gives D_W^dag (the adjoint hop of dwf.dhop)."""
    h = dwf.dhop(U, psi[:, :, :, :, None], dag=dag)[:, :, :, :, 0]
    return (mass + 4.0) * psi - 0.5 * h


def wilson_normal(U, psi, mass):
    """D_W^dag D_W psi."""
    return wilson(U, wilson(U, psi, mass), mass, dag=True)


def gamma5_project(phi, sign):
    """(1 + sign gamma_5)/2 phi on a 4D field."""
    return 0.5 * (phi + sign * dwf.apply_spin(dwf.GAMMA5, phi))


def basis4(U, etas, mass, lo, hi, order, block):
    """The 4D block basis: each eta filtered by T_order(x(D_W^dag D_W)) on
    [lo, hi], the first half projected with (1 + gamma_5)/2, the rest with
    (1 - gamma_5)/2, block orthonormalised per chirality."""
    appA = lambda w: wilson_normal(U, w, mass)
    raw = [cheby.cheby_filter(appA, e, order, lo, hi) for e in etas]
    nb = len(raw)
    half = nb // 2
    vecs = [gamma5_project(v, +1) for v in raw[:half]] + [gamma5_project(v, -1) for v in raw[half:]]
    return coarse.block_orthonormalise(vecs, block, [list(range(half)), list(range(half, nb))])


def hop4_term(U, phi, block, d):
    """The d-th term of -1/2 D_hop on 4D blocks: d = 1+2mu (2+2mu) the hop from
    x+mu (x-mu) kept at sites on the +mu (-mu) face of their block; d = 0 the
    sum of the hops that stay inside the block."""
    L = dwf.lattice_dims(phi)
    p5 = phi[:, :, :, :, None]
    if d > 0:
        mu, sgn = (d - 1) // 2, (+1 if (d - 1) % 2 == 0 else -1)
        h = -0.5 * dwf.dhop_direction(U, p5, mu, sgn)[:, :, :, :, 0]
        return coarse.face_mask(L, block, mu, sgn)[..., None, None] * h
    out = np.zeros_like(phi)
    for mu in range(4):
        for sgn in (+1, -1):
            h = -0.5 * dwf.dhop_direction(U, p5, mu, sgn)[:, :, :, :, 0]
            out += (1 - coarse.face_mask(L, block, mu, sgn))[..., None, None] * h
    return out


def coarse_build4(U, basis, block):
    """B[d][x][j, k] = <phi_j^x, (-1/2 D_hop)^(d) phi_k^(x+d)> (Eq. 18 for the
    hopping part of D_W): shape (9, Tc, Zc, Yc, Xc, nb, nb)."""
    L = dwf.lattice_dims(basis[0])
    Lc = coarse.coarse_dims(L, block)
    nb = len(basis)
    B = np.zeros((coarse.NDIR, Lc[3], Lc[2], Lc[1], Lc[0], nb, nb), complex)
    for k, phk in enumerate(basis):
        for d in range(coarse.NDIR):
            W = hop4_term(U, phk, block, d)
            for j, phj in enumerate(basis):
                B[d, ..., j, k] = coarse.block_inner(phj, W, block)
    return B


# ---------------------------------------------------------------- level 1
def chirality(nb, nplus):
    return np.array([1.0] * nplus + [-1.0] * (nb - nplus))


def fifth_scalar(Ls, M5, mf, chi):
    """The Ls x Ls fifth-dimension matrix of Eq. (4) on one chirality: the
    P_+ (chi = +1) or P_- (chi = -1) diagonal entry of dwf.fifth_dim_matrix."""
    K = dwf.fifth_dim_matrix(Ls, M5, mf)
    return K[:, :, 0, 0] if chi > 0 else K[:, :, 2, 2]


def restrict1(basis, psi, block):
    """P1^dag psi: v(x_c, k, s) = sum_{x in block x_c} phi_k(x)^dag psi(x, s)."""
    Ls = psi.shape[4]
    out = np.stack([np.stack([coarse.block_inner(phi, psi[:, :, :, :, s], block) for s in range(Ls)], axis=-1)
                    for phi in basis], axis=-2)
    return out


def prolong1(basis, v, block):
    """P1 v: psi(x, s) = sum_k phi_k(x) v(x_c(x), k, s)."""
    Ls = v.shape[-1]
    phi0 = basis[0]
    out = np.zeros(phi0.shape[:4] + (Ls,) + phi0.shape[4:], complex)
    for k, phi in enumerate(basis):
        for s in range(Ls):
            out[:, :, :, :, s] += coarse._expand(v[..., k, s], block, phi.shape) * phi
    return out


def level1_hop(B, v, d=None):
    """sum_d B_d(x) v(x+d) on every s (or the single term d)."""
    out = np.zeros_like(v)
    for dd in (range(coarse.NDIR) if d is None else [d]):
        out += np.einsum("...jk,...ks->...js", B[dd], coarse.coarse_neighbour(v, dd))
    return out


def level1_fifth(v, M5, mf, nplus):
    """K_chi_k applied on the fifth dimension of every basis index k."""
    nb, Ls = v.shape[-2], v.shape[-1]
    out = np.zeros_like(v)
    for k, chi in enumerate(chirality(nb, nplus)):
        out[..., k, :] = np.einsum("st,...t->...s", fifth_scalar(Ls, M5, mf, chi), v[..., k, :])
    return out


def gamma5_1(v, nplus):
    """Gamma5_1 v = chi_k v(x, k, Ls-1-s)."""
    chi = chirality(v.shape[-2], nplus)
    return chi[:, None] * v[..., ::-1]


def level1_apply(B, v, M5, mf, nplus):
    """M_1 v = K_chi v + sum_d B_d v(x+d)."""
    return level1_fifth(v, M5, mf, nplus) + level1_hop(B, v)


def level1_herm(B, v, M5, mf, nplus):
    """H_1 v = Gamma5_1 M_1 v."""
    return gamma5_1(level1_apply(B, v, M5, mf, nplus), nplus)


def chiral_project1(v, sign, nplus):
    """(1 + sign Gamma5_1)/2 v."""
    return 0.5 * (v + sign * gamma5_1(v, nplus))


# ---------------------------------------------------------------- level 2
def basis2(B, etas, M5, mf, nplus4, lo, hi, order):
    """Level-2 basis: each level-1 eta filtered by T_order(x(H_1^2)) on
    [lo, hi], the first half projected with (1 + Gamma5_1)/2, the rest with
    (1 - Gamma5_1)/2, orthonormalised per level-1 site and chirality."""
    appA = lambda w: level1_herm(B, level1_herm(B, w, M5, mf, nplus4), M5, mf, nplus4)
    raw = [cheby.cheby_filter(appA, e, order, lo, hi) for e in etas]
    nb = len(raw)
    half = nb // 2
    vecs = [chiral_project1(v, +1, nplus4) for v in raw[:half]] + \
           [chiral_project1(v, -1, nplus4) for v in raw[half:]]
    return coarse.block_orthonormalise(vecs, SITE, [list(range(half)), list(range(half, nb))])


def level1_term(B, v, d, M5, mf, nplus):
    """The d-th term of H_1: Gamma5_1 B_d v(x+d), plus Gamma5_1 K v for d = 0."""
    t = level1_hop(B, v, d)
    if d == 0:
        t = t + level1_fifth(v, M5, mf, nplus)
    return gamma5_1(t, nplus)


def coarse_build2(B, basis, M5, mf, nplus4):
    """A2[d][x][i, j] = <Phi_i^x, H_1^(d) Phi_j^(x+d)>: shape (9, Tc, Zc, Yc, Xc, nb2, nb2)."""
    nb = len(basis)
    sh = basis[0].shape[:4]
    A = np.zeros((coarse.NDIR,) + sh + (nb, nb), complex)
    for j, phj in enumerate(basis):
        for d in range(coarse.NDIR):
            W = level1_term(B, phj, d, M5, mf, nplus4)
            for i, phi in enumerate(basis):
                A[d, ..., i, j] = coarse.block_inner(phi, W, SITE)
    return A


def restrict2(basis, v):
    return np.stack([coarse.block_inner(phi, v, SITE) for phi in basis], axis=-1)


def prolong2(basis, e):
    out = np.zeros_like(basis[0])
    for i, phi in enumerate(basis):
        out += e[..., i][..., None, None] * phi
    return out


# ---------------------------------------------------------------- W-cycle
class Hybrid:
    """The three levels of Algorithm F with the parameters of its solve."""

    def __init__(self, U, M5, mf, block, b4, B, b2, A2, smooth=(0.5, 60.0, 12), smooth1=(0.5, 60.0, 0),
                 kcycle=2, coarse_tol=0.02, coarse_maxiter=500):
        self.U, self.M5, self.mf, self.block = U, M5, mf, block
        self.b4, self.B, self.b2, self.A2 = b4, B, b2, A2
        self.nplus4 = len(b4) // 2
        self.smooth, self.smooth1 = smooth, smooth1
        self.kcycle, self.coarse_tol, self.coarse_maxiter = kcycle, coarse_tol, coarse_maxiter
        if kcycle > 1 and smooth1[2] == 0:
            # without a level-1 smoother the preconditioner is K = P2 A_2^-1 P2^dag
            # and K H_1 K = K (A_2 = P2^dag H_1 P2), so the second GCR direction
            # vanishes in exact arithmetic and only rounding would be amplified
            raise ValueError("kcycle > 1 needs a level-1 smoother")

    def H1(self, v):
        return level1_herm(self.B, v, self.M5, self.mf, self.nplus4)


class Counter(mg.MGCounter):
    def __init__(self):
        super().__init__()
        self.level1 = 0
        self.solves2 = 0


def level1_vcycle(h, r, cnt):
    """V(1,1) on level 1 (Eqs. 26-28 with M = H_1): smoother, coarse-coarse
    correction P2 A_2^-1 P2^dag, smoother."""
    a, b, N = h.smooth1
    x = np.zeros_like(r)
    if N > 0:
        x, n = cheby.smoother_apply(h.H1, h.H1, r, a, b, N)
        cnt.level1 += n
    r1 = r - h.H1(x) if N > 0 else r
    cnt.level1 += 1 if N > 0 else 0
    e2, it = coarse.coarse_cgnr(h.A2, restrict2(h.b2, r1), h.coarse_tol, h.coarse_maxiter)
    cnt.coarse += it
    cnt.solves2 += 1
    x = x + prolong2(h.b2, e2)
    if N > 0:
        r2 = r - h.H1(x)
        s2, n = cheby.smoother_apply(h.H1, h.H1, r2, a, b, N)
        cnt.level1 += 1 + n
        x = x + s2
    return x


def level1_solve(h, r, cnt):
    """kcycle iterations of flexible GCR on H_1 e = r from e = 0 with no
    tolerance test (the fixed W-cycle): z = V_1(res), w = H_1 z orthogonalised
    against the earlier w, e += alpha z, res -= alpha w."""
    e = np.zeros_like(r)
    if dwf.norm2(r) == 0:
        return e
    res = r.copy()
    zs, ws = [], []
    for _ in range(h.kcycle):
        z = level1_vcycle(h, res, cnt)
        w = h.H1(z)
        cnt.level1 += 1
        for zj, wj in zip(zs, ws):
            beta = dwf.inner(wj, w) / dwf.norm2(wj)
            w = w - beta * wj
            z = z - beta * zj
        alpha = dwf.inner(w, res) / dwf.norm2(w)
        e = e + alpha * z
        res = res - alpha * w
        zs.append(z)
        ws.append(w)
    return e


def hybrid_vcycle(h, r0, cnt):
    """The fine V(1,1) (Eqs. 26-28 with M = H_DW) whose coarse correction is
    P1 e, e from the level-1 W-cycle solve of H_1 e = P1^dag r1."""
    apply_H = lambda v: dwf.hdw(h.U, v, h.M5, h.mf)
    a, b, N = h.smooth
    x1, n = cheby.smoother_apply(apply_H, apply_H, r0, a, b, N)
    cnt.fine += n
    r1 = r0 - apply_H(x1)
    cnt.fine += 1
    e1 = level1_solve(h, restrict1(h.b4, r1, h.block), cnt)
    x2 = x1 + prolong1(h.b4, e1, h.block)
    r2 = r0 - apply_H(x2)
    cnt.fine += 1
    s2, n = cheby.smoother_apply(apply_H, apply_H, r2, a, b, N)
    cnt.fine += n
    return x2 + s2


def hybrid_solve(h, b, tol, maxiter=200, nkrylov=8):
    """Algorithm F solve of D_DW x = b: flexible GCR on H_DW x = Gamma_5 b with
    the hybrid V(1,1) preconditioner; stops when ||b - D_DW x|| / ||b|| <= tol."""
    apply_H = lambda v: dwf.hdw(h.U, v, h.M5, h.mf)
    cnt = Counter()
    pre = lambda r: hybrid_vcycle(h, r, cnt)
    x, it, hist = mg.pgcr(apply_H, dwf.gamma5_r5(b), pre, tol, maxiter, nkrylov, cnt)
    return x, it, hist, cnt
