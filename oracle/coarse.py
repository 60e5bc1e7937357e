"""Blocking, chirality projection and the little Dirac operator in FP64
(oracle; test infrastructure only).

Paper: arXiv:2103.05034.
  Sec. 3.1, Eq. (14): phi^b_k(x) = phi_k(x) for x in block b, 0 otherwise
  Sec. 3.1, Eq. (18): A^{ab}_{jk} = <phi^a_j | M | phi^b_k>, with restrictor
           P^dag = <phi^b_k| and prolongator P = |phi^b_k>; A is nearest
           neighbour because well separated blocks do not connect through M
  Sec. 3.4 (end): the basis is projected with (1 +- Gamma_5)/2 for the five
           dimensional coarsening, so Gamma_5 is a sign on the coarse space
  Sec. 4, Table 1: HDCR coarsens M = H_DW with blocks spanning all of Ls

  Sec. 3.5 (coarse space deflation) and the setup table of Sec. 5: the coarse
           solve is CG on the normal equations deflated with Lanczos
           eigenvectors, the Lanczos run on a Chebyshev polynomial of the
           operator (the high-order polynomial grows fast outside [-1, 1]
           and so enhances the wanted low modes); the vectors serve as a
           basis in which the operator is diagonal
  Sec. 5.3 (the 48^3 study): a red-black solver on the coarse space; the
           nearest-neighbour stencil couples each coarse site to itself and
           to sites of the other coarse parity only, so A = [[A_ee, A_eo],
           [A_oe, A_oo]] with block-diagonal A_ee, A_oo (the nb x nb self
           terms) and the even Schur complement S = A_ee - A_eo A_oo^-1 A_oe

Readings:
  * Coarse deflation: Lanczos with full reorthogonalisation on
    B = T_n(y(A^2)), y(t) = 2 (t - lam_lo) / (lam_max - lam_lo) - 1 (n even,
    so the modes of A^2 below lam_lo are B's largest), for nk steps from a
    Gaussian start; the nev Ritz vectors of B's largest Ritz values are then
    diagonalised with A^2 itself (Rayleigh-Ritz), giving pairs (theta_i,
    v_i); the deflated coarse CG starts from sum_i v_i <v_i, b> / theta_i.
  * Blocks are b_x x b_y x b_z x b_t x Ls (the whole fifth dimension).
  * The paper implies P^dag P = 1 but does not say how; each (block,
    chirality) group is orthonormalised by modified Gram-Schmidt, applied
    twice, in ascending vector order.
  * Coarse stencil directions: d = 0 (self), then +x, -x, +y, -y, +z, -z,
    +t, -t.  A_d(x)_{jk} = <phi^x_j, H^(d) phi^{x+d}_k>, H^(d) the part of
    H_DW that carries block x+d into block x.  When the coarse extent is 1 or
    2 in a direction, several d reach the same block; they stay separate
    terms of the stencil and their sum is the dense matrix element.
"""
from __future__ import annotations

import numpy as np

from . import dwf

NDIR = 9


def coarse_dims(L, block):
    return tuple(L[m] // block[m] for m in range(4))


def to_blocks(psi, block):
    """(T,Z,Y,X,Ls,4,3) -> (Tc,Zc,Yc,Xc, block dof)."""
    T, Z, Y, X = psi.shape[:4]
    bx, by, bz, bt = block
    rest = psi.shape[4:]
    v = psi.reshape((T // bt, bt, Z // bz, bz, Y // by, by, X // bx, bx) + rest)
    v = v.transpose((0, 2, 4, 6, 1, 3, 5, 7) + tuple(range(8, 8 + len(rest))))
    return v.reshape((T // bt, Z // bz, Y // by, X // bx, -1))


def block_inner(a, b, block):
    """<a|_block |b>_block for every block: (Tc,Zc,Yc,Xc)."""
    return np.einsum("...i,...i->...", to_blocks(a, block).conj(), to_blocks(b, block))


def block_index_field(L, block):
    """Per 4D site the (tc, zc, yc, xc) of its block, and masks of block faces."""
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly),
                             np.arange(Lx), indexing="ij")
    return (x, y, z, t)


def face_mask(L, block, mu, sign):
    """1 at sites whose neighbour in direction sign*mu lies in another block
    (or, for a coarse extent of one, wraps around into the same block)."""
    coords = block_index_field(L, block)
    c = coords[mu] % block[mu]
    if sign > 0:
        m = (c == block[mu] - 1)
    else:
        m = (c == 0)
    return m.astype(float)


def chiral_project(phi, sign):
    """(1 + sign Gamma_5)/2 phi."""
    return 0.5 * (phi + sign * dwf.gamma5_r5(phi))


def block_orthonormalise(vecs, block, groups):
    """Modified Gram-Schmidt, twice, within each block and each group of
    vector indices, in ascending order.  Returns new list."""
    out = [v.copy() for v in vecs]
    for grp in groups:
        for _pass in range(2):
            for ii, i in enumerate(grp):
                v = out[i]
                for j in grp[:ii]:
                    c = block_inner(out[j], v, block)
                    v = v - _expand(c, block, v.shape) * out[j]
                nrm = np.sqrt(block_inner(v, v, block).real)
                if np.min(nrm) < 1e-12:
                    raise ValueError("basis vector vanished on a block")
                out[i] = v / _expand(nrm, block, v.shape)
    return out


def _expand(c, block, shape):
    """Broadcast a per-block scalar (Tc,Zc,Yc,Xc) to a fine field shape."""
    bx, by, bz, bt = block
    e = np.repeat(np.repeat(np.repeat(np.repeat(c, bt, 0), bz, 1), by, 2), bx, 3)
    return e.reshape(e.shape + (1,) * (len(shape) - 4))


def restrict(basis, psi, block):
    """P^dag psi: coarse vector (Tc,Zc,Yc,Xc,nb)."""
    return np.stack([block_inner(phi, psi, block) for phi in basis], axis=-1)


def prolong(basis, vc, block):
    """P v_c = sum_k phi^b_k v_c(b)_k."""
    out = np.zeros_like(basis[0])
    for k, phi in enumerate(basis):
        out += _expand(vc[..., k], block, phi.shape) * phi
    return out


def coarse_build(U, basis, block, M5, mf):
    """The 9-point stencil A[d] of H_DW on the block basis:
    returns (9, Tc, Zc, Yc, Xc, nb, nb) with A[d][x][j, k]."""
    L = dwf.lattice_dims(basis[0])
    nb = len(basis)
    Lc = coarse_dims(L, block)
    A = np.zeros((NDIR, Lc[3], Lc[2], Lc[1], Lc[0], nb, nb), complex)
    Ls = basis[0].shape[4]
    Kd = dwf.k_dense(dwf.fifth_dim_matrix(Ls, M5, mf))
    for k, phi in enumerate(basis):
        self_part = dwf.apply_dense_sitelocal(Kd, phi)
        parts = {}
        for mu in range(4):
            for sgn in (+1, -1):
                h = -0.5 * dwf.dhop_direction(U, phi, mu, sgn)
                fm = face_mask(L, block, mu, sgn)[..., None, None, None]
                parts[(mu, sgn)] = dwf.gamma5_r5(fm * h)
                self_part = self_part + (1 - fm) * h
        self_part = dwf.gamma5_r5(self_part)
        for j, phj in enumerate(basis):
            A[0, ..., j, k] = block_inner(phj, self_part, block)
            for mu in range(4):
                for sgn in (+1, -1):
                    d = 1 + 2 * mu + (0 if sgn > 0 else 1)
                    A[d, ..., j, k] = block_inner(phj, parts[(mu, sgn)], block)
    return A


def coarse_neighbour(vc, d):
    """v_c(x + d) on the periodic coarse lattice."""
    if d == 0:
        return vc
    mu, sgn = (d - 1) // 2, (+1 if (d - 1) % 2 == 0 else -1)
    return np.roll(vc, -sgn, axis=(3, 2, 1, 0)[mu])


def coarse_apply(A, vc):
    """out(x) = sum_d A_d(x) v(x + d)."""
    out = np.zeros_like(vc)
    for d in range(NDIR):
        out += np.einsum("...jk,...k->...j", A[d], coarse_neighbour(vc, d))
    return out


def coarse_dense_from_stencil(A):
    """The stencil as a dense matrix on (coarse site, basis index)."""
    nd, Tc, Zc, Yc, Xc, nb, _ = A.shape
    n = Tc * Zc * Yc * Xc * nb
    D = np.zeros((n, n), complex)
    for i in range(n):
        e = np.zeros(n, complex)
        e[i] = 1
        D[:, i] = coarse_apply(A, e.reshape(Tc, Zc, Yc, Xc, nb)).ravel()
    return D


def coarse_dense_bruteforce(U, basis, block, M5, mf):
    """P^dag H_DW P by applying H_DW to every block basis vector phi^b_k."""
    L = dwf.lattice_dims(basis[0])
    Lc = coarse_dims(L, block)
    nb = len(basis)
    nc = Lc[0] * Lc[1] * Lc[2] * Lc[3]
    D = np.zeros((nc * nb, nc * nb), complex)
    for c in range(nc):
        sel = np.zeros(nc)
        sel[c] = 1.0
        sel = sel.reshape(Lc[3], Lc[2], Lc[1], Lc[0])
        for k, phi in enumerate(basis):
            col = dwf.hdw(U, _expand(sel, block, phi.shape) * phi, M5, mf)
            D[:, c * nb + k] = restrict(basis, col, block).ravel()
    return D


def coarse_cgnr(A, rc, tol, maxiter):
    """CG on A^2 e = A r_c for the hermitian coarse operator; stops when the
    normal-equation residual falls below tol times its initial value."""
    b = coarse_apply(A, rc)
    x = np.zeros_like(rc)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    bb = rr
    it = 0
    while it < maxiter and rr > tol * tol * bb:
        Ap = coarse_apply(A, coarse_apply(A, p))
        alpha = rr / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


def coarse_parity_mask(Lc_shape):
    """1 on even coarse sites ((xc + yc + zc + tc) even) of a (Tc,Zc,Yc,Xc) lattice."""
    t, z, y, x = np.indices(Lc_shape)
    return ((x + y + z + t) % 2 == 0).astype(float)


def coarse_rb_solve(A, rc, tol, maxiter):
    """Red-black solve of A e = r_c (Sec. 5.3): CG on S^2 e_e = S r'_e with
    the even Schur complement S (hermitian when A is), r'_e = r_e - A_eo
    A_oo^-1 r_o, then e_o = A_oo^-1 (r_o - A_oe e_e).  Stops when the
    normal-equation residual falls below tol times its initial value.  Needs
    even coarse extents (otherwise the stencil couples a parity to itself:
    ValueError).  Returns (e, iterations)."""
    shape = A.shape[1:5]
    if any(n % 2 for n in shape):
        raise ValueError("red-black coarse solve needs even coarse extents")
    me = coarse_parity_mask(shape)[..., None]
    mo = 1.0 - me
    self_inv = np.linalg.inv(A[0])

    def off(v):  # sum over the eight neighbour terms
        out = np.zeros_like(v)
        for d in range(1, NDIR):
            out += np.einsum("...jk,...k->...j", A[d], coarse_neighbour(v, d))
        return out

    def self_apply(M, v):
        return np.einsum("...jk,...k->...j", M, v)

    def schur(v):  # S v on even sites (v even)
        t = mo * self_apply(self_inv, mo * off(v))
        return me * (self_apply(A[0], v) - off(t))

    r_e, r_o = me * rc, mo * rc
    rp = r_e - me * off(mo * self_apply(self_inv, r_o))
    b = schur(rp)
    x = np.zeros_like(rc)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    bb = rr
    it = 0
    while it < maxiter and rr > tol * tol * bb:
        Ap = schur(schur(p))
        alpha = rr / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    e_o = mo * self_apply(self_inv, r_o - mo * off(x))
    return x + e_o, it


def cheby_lanczos(apply_AA, v0, nev, nk, order, lam_lo, lam_max):
    """Chebyshev-preconditioned Lanczos (reading above) on the hermitian
    positive operator A^2 (apply_AA): returns (theta, V), nev Rayleigh-Ritz
    pairs for its lowest modes, V a list of orthonormal vectors."""
    if order % 2:
        raise ValueError("even Chebyshev order")
    from .cheby import cheby_filter
    B = lambda v: cheby_filter(apply_AA, v, order, lam_lo, lam_max)
    Q = [v0 / np.sqrt(np.vdot(v0, v0).real)]
    alpha, beta = [], []
    for j in range(nk):
        w = B(Q[j])
        a = np.vdot(Q[j], w).real
        alpha.append(a)
        w = w - a * Q[j] - (beta[j - 1] * Q[j - 1] if j > 0 else 0)
        for q in Q:  # full reorthogonalisation
            w = w - np.vdot(q, w) * q
        b = np.sqrt(np.vdot(w, w).real)
        if j == nk - 1 or b < 1e-14:
            break
        beta.append(b)
        Q.append(w / b)
    k = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:k - 1], 1) + np.diag(beta[:k - 1], -1)
    mu, S = np.linalg.eigh(T)
    top = np.argsort(mu)[::-1][:nev]  # B's largest: A^2's lowest
    W = [sum(S[i, t] * Q[i] for i in range(k)) for t in top]
    # Rayleigh-Ritz with A^2 on span(W)
    H = np.array([[np.vdot(wi, apply_AA(wj)) for wj in W] for wi in W])
    th, C = np.linalg.eigh(0.5 * (H + H.conj().T))
    V = [sum(C[i, t] * W[i] for i in range(len(W))) for t in range(len(W))]
    return th, V


def coarse_deflated_cgnr(A, rc, theta, V, tol, maxiter):
    """CG on A^2 e = A r_c (as coarse_cgnr) started from the deflation guess
    e_0 = sum_i v_i <v_i, A r_c> / theta_i; stops when the normal-equation
    residual falls below tol times that of the zero start."""
    b = coarse_apply(A, rc)
    x = np.zeros_like(rc)
    for th, v in zip(theta, V):
        x = x + v * (np.vdot(v, b) / th)
    AA = lambda u: coarse_apply(A, coarse_apply(A, u))
    r = b - AA(x)
    p = r.copy()
    rr = np.vdot(r, r).real
    bb = np.vdot(b, b).real
    it = 0
    while it < maxiter and rr > tol * tol * bb:
        Ap = AA(p)
        alpha = rr / np.vdot(p, Ap).real
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it
