"""Pins of the FP64 oracle's operators (Sec. 2 of arXiv:2103.05034) against
closed forms, identities and plain dense linear algebra."""
import numpy as np
import pytest

import synth
from oracle import dwf, krylov

M5 = 1.8


def rand_field(L, Ls, seed):
    return synth.gaussian_spinor(L, Ls, seed)


def test_gamma_algebra():
    G = dwf.GAMMA
    for m in range(4):
        assert np.allclose(G[m], G[m].conj().T)
        for n in range(4):
            ac = G[m] @ G[n] + G[n] @ G[m]
            assert np.allclose(ac, 2 * (m == n) * np.eye(4))
    assert np.allclose(dwf.GAMMA5, np.diag([1, 1, -1, -1]))
    for m in range(4):
        assert np.allclose(dwf.GAMMA5 @ G[m] + G[m] @ dwf.GAMMA5, 0)


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 3), (3, 1, 1, 5)])
def test_free_field_plane_wave_dhop(n):
    """U = 1: D_hop e^{ipx} chi = e^{ipx} sum_mu (2 cos p_mu - 2 i gamma_mu sin p_mu) chi."""
    L = (4, 4, 4, 8)
    Ls = 3
    p = [2 * np.pi * n[m] / L[m] for m in range(4)]
    U = np.zeros((L[3], L[2], L[1], L[0], 4, 3, 3), complex)
    U[...] = np.eye(3)
    chi = synth.complex_gaussian(7, (Ls, 4, 3))
    t, z, y, x = np.meshgrid(*[np.arange(L[a]) for a in (3, 2, 1, 0)], indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    psi = phase[..., None, None, None] * chi
    got = dwf.dhop(U, psi)
    Dp = sum(2 * np.cos(p[m]) * np.eye(4) - 2j * np.sin(p[m]) * dwf.GAMMA[m] for m in range(4))
    want = phase[..., None, None, None] * np.einsum("ij,sjc->sic", Dp, chi)
    assert np.allclose(got, want, atol=1e-12)


def test_free_field_dpar_eigenvalues():
    """D_par(p) = 5 - M5 - sum cos p - (-i) sum gamma sin p has eigenvalues
    5 - M5 - sum cos p_mu +- i sqrt(sum sin^2 p_mu) (the 4D part of the free
    5D Wilson spectrum quoted in Sec. 2.1)."""
    L = (4, 4, 4, 8)
    n = (1, 2, 0, 3)
    p = [2 * np.pi * n[m] / L[m] for m in range(4)]
    U = np.zeros((L[3], L[2], L[1], L[0], 4, 3, 3), complex)
    U[...] = np.eye(3)
    t, z, y, x = np.meshgrid(*[np.arange(L[a]) for a in (3, 2, 1, 0)], indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    # build the 4x4 spin matrix of D_par on this momentum by applying it to basis spinors
    Dm = np.zeros((4, 4), complex)
    for j in range(4):
        chi = np.zeros((1, 4, 3), complex)
        chi[0, j, 0] = 1
        psi = phase[..., None, None, None] * chi
        out = (5 - M5) * psi - 0.5 * dwf.dhop(U, psi)
        Dm[:, j] = out[0, 0, 0, 0, 0, :, 0] / phase[0, 0, 0, 0]
    ev = np.linalg.eigvals(Dm)
    ev = ev[np.argsort(ev.imag)]
    re = 5 - M5 - sum(np.cos(p))
    im = np.sqrt(sum(np.sin(pp) ** 2 for pp in p))
    want = np.array([re - 1j * im, re - 1j * im, re + 1j * im, re + 1j * im])
    assert np.allclose(ev, want, atol=1e-12)


@pytest.fixture(scope="module")
def small():
    L = (4, 4, 4, 4)
    Ls = 4
    U = synth.random_gauge(L, 0.5, 11)
    return L, Ls, U


def test_links_are_su3(small):
    L, Ls, U = small
    UdU = np.einsum("...ji,...jk->...ik", U.conj(), U)
    assert np.allclose(UdU, np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(U), 1, atol=1e-13)
    Us = synth.random_gauge((4, 4, 4, 4), 0.5, 11, ape_steps=2)
    assert np.allclose(np.einsum("...ji,...jk->...ik", Us.conj(), Us), np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(Us), 1, atol=1e-13)


def test_adjoint_identity(small):
    L, Ls, U = small
    x = rand_field(L, Ls, 1)
    y = rand_field(L, Ls, 2)
    for mf in (0.01, 0.3):
        lhs = dwf.inner(x, dwf.ddw(U, y, M5, mf))
        rhs = dwf.inner(dwf.ddw(U, x, M5, mf, dag=True), y)
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    lhs = dwf.inner(x, dwf.dhop(U, y))
    rhs = dwf.inner(dwf.dhop(U, x, dag=True), y)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_gamma5_hermiticity(small):
    """Gamma_5 D_DW Gamma_5 = D_DW^dag, so H_DW = Gamma_5 D_DW is hermitian (Eq. 6)."""
    L, Ls, U = small
    x = rand_field(L, Ls, 3)
    y = rand_field(L, Ls, 4)
    mf = 0.05
    lhs = dwf.inner(x, dwf.gamma5_r5(dwf.ddw(U, dwf.gamma5_r5(y), M5, mf)))
    rhs = dwf.inner(dwf.ddw(U, x, M5, mf), y)
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    a = dwf.inner(x, dwf.hdw(U, y, M5, mf))
    b = dwf.inner(dwf.hdw(U, x, M5, mf), y)
    assert abs(a - b) < 1e-11 * abs(a)


def test_gauge_covariance(small):
    """D[U^g](g psi) = g D[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag."""
    L, Ls, U = small
    g = synth.random_gauge_transform(L, 99)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ dwf.dagger(dwf.shift(g, mu, +1))
    psi = rand_field(L, Ls, 5)
    gpsi = dwf.apply_color(g, psi)
    lhs = dwf.ddw(Ug, gpsi, M5, 0.1)
    rhs = dwf.apply_color(g, dwf.ddw(U, psi, M5, 0.1))
    assert np.allclose(lhs, rhs, atol=1e-12)


def closed_form_mplus_inv(Ls, d, m):
    """(M_+^-1)_{s,s'} = d^{-1-j} (s<s' ? -m : 1) / (1 + m d^{-Ls}), j = (s-s') mod Ls,
    derived from M_+ = d - L' with the twisted cyclic shift L' (L'^Ls = -m)."""
    A = np.zeros((Ls, Ls))
    for s in range(Ls):
        for sp in range(Ls):
            j = (s - sp) % Ls
            A[s, sp] = d ** (-1 - j) * (-m if s < sp else 1.0) / (1 + m * d ** (-Ls))
    return A


@pytest.mark.parametrize("Ls,mf", [(4, 0.01), (8, 0.3), (16, 0.01), (24, 0.00078)])
def test_mooee_inverse_closed_form(Ls, mf):
    K = dwf.fifth_dim_matrix(Ls, M5, mf)
    Kinv = np.linalg.inv(dwf.k_dense(K)).reshape(Ls, 4, Ls, 4)
    d = 5 - M5
    Ap = closed_form_mplus_inv(Ls, d, mf)
    # chirality + lives on spins 0,1 (gamma_5 = +1); chirality - is the transpose
    for sp in range(4):
        blk = Kinv[:, sp, :, sp].real
        want = Ap if sp < 2 else Ap.T
        assert np.allclose(blk, want, rtol=1e-12, atol=1e-15)
    assert np.allclose(Kinv.imag, 0)


def test_mooee_inv_roundtrip(small):
    L, Ls, U = small
    psi = rand_field(L, Ls, 6)
    for dag in (False, True):
        back = dwf.mooee(dwf.mooee_inv(psi, M5, 0.02, dag=dag), M5, 0.02, dag=dag)
        assert np.allclose(back, psi, atol=1e-12)


def dense_operator(apply, shape):
    n = int(np.prod(shape))
    A = np.zeros((n, n), complex)
    for i in range(n):
        e = np.zeros(n, complex)
        e[i] = 1
        A[:, i] = apply(e.reshape(shape)).ravel()
    return A


@pytest.fixture(scope="module")
def tiny():
    L = (2, 2, 2, 2)
    Ls = 4
    U = synth.random_gauge(L, 0.7, 21)
    shape = (2, 2, 2, 2, Ls, 4, 3)
    D = dense_operator(lambda v: dwf.ddw(U, v, M5, 0.05), shape)
    return L, Ls, U, shape, D


def test_schur_complement_dense(tiny):
    """M_pc equals the Schur complement D_ee - D_eo D_oo^-1 D_oe of the dense D_DW."""
    L, Ls, U, shape, D = tiny
    mask = np.broadcast_to(dwf.parity_mask(L)[..., None, None, None], shape).ravel() > 0.5
    e, o = np.where(mask)[0], np.where(~mask)[0]
    S = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    v = dwf.project_parity(rand_field(L, Ls, 8), L, 0)
    got = dwf.mpc(U, v, M5, 0.05).ravel()
    want = np.zeros_like(got)
    want[e] = S @ v.ravel()[e]
    assert np.allclose(got, want, atol=1e-12)
    gotd = dwf.mpc_dag(U, v, M5, 0.05).ravel()
    wantd = np.zeros_like(gotd)
    wantd[e] = S.conj().T @ v.ravel()[e]
    assert np.allclose(gotd, wantd, atol=1e-12)


def test_rbcg_matches_dense_solve(tiny):
    L, Ls, U, shape, D = tiny
    b = rand_field(L, Ls, 9)
    x_dense = np.linalg.solve(D, b.ravel()).reshape(shape)
    x, it, _ = krylov.rbcg_solve(U, b, M5, 0.05, 1e-13)
    assert np.linalg.norm(x - x_dense) / np.linalg.norm(x_dense) < 1e-10
    assert krylov.true_residual(U, x, b, M5, 0.05) < 1e-11


def test_second_schur_form_matches_dense_solve(tiny):
    """Table 5's second red-black form, (1 - M_ee^-1 M_eo M_oo^-1 M_oe), is
    M_ee^-1 times the Schur complement, and its CGNR reaches the dense
    solution."""
    L, Ls, U, shape, D = tiny
    mask = np.broadcast_to(dwf.parity_mask(L)[..., None, None, None], shape).ravel() > 0.5
    e, o = np.where(mask)[0], np.where(~mask)[0]
    S = D[np.ix_(e, e)] - D[np.ix_(e, o)] @ np.linalg.solve(D[np.ix_(o, o)], D[np.ix_(o, e)])
    S2 = np.linalg.solve(D[np.ix_(e, e)], S)
    v = dwf.project_parity(rand_field(L, Ls, 11), L, 0)
    assert np.allclose(dwf.mpc2(U, v, M5, 0.05).ravel()[e], S2 @ v.ravel()[e], atol=1e-12)
    assert np.allclose(dwf.mpc2_dag(U, v, M5, 0.05).ravel()[e], S2.conj().T @ v.ravel()[e], atol=1e-12)
    b = rand_field(L, Ls, 12)
    x_dense = np.linalg.solve(D, b.ravel()).reshape(shape)
    x, it, _ = krylov.rbcg2_solve(U, b, M5, 0.05, 1e-13)
    assert np.linalg.norm(x - x_dense) / np.linalg.norm(x_dense) < 1e-10


def test_cgnr_matches_dense_solve(tiny):
    """CG on D^dag D x = D^dag b (the unpreconditioned baseline of Sec. 5.1)
    reaches the dense solution, in more iterations than the red-black solve
    (the Schur complement is better conditioned)."""
    L, Ls, U, shape, D = tiny
    b = rand_field(L, Ls, 10)
    x_dense = np.linalg.solve(D, b.ravel()).reshape(shape)
    rhs = dwf.ddw(U, b, M5, 0.05, dag=True)
    x, it, _ = krylov.cg(lambda v: dwf.mdagm(U, v, M5, 0.05), rhs, 1e-13, 10000)
    assert np.linalg.norm(x - x_dense) / np.linalg.norm(x_dense) < 1e-10
    _, it_rb, _ = krylov.rbcg_solve(U, b, M5, 0.05, 1e-13)
    assert it > it_rb


def test_hdw_spectrum_real_and_squares(tiny):
    """H_DW is hermitian; its squared spectrum is that of D^dag D."""
    L, Ls, U, shape, D = tiny
    G = dense_operator(dwf.gamma5_r5, shape)
    H = G @ D
    assert np.allclose(H, H.conj().T, atol=1e-12)
    ev = np.sort(np.linalg.eigvalsh(H) ** 2)
    sv = np.sort(np.linalg.eigvalsh(D.conj().T @ D))
    assert np.allclose(ev, sv, rtol=1e-9, atol=1e-12)


def test_power_method(tiny):
    L, Ls, U, shape, D = tiny
    A = D.conj().T @ D
    lmax = np.linalg.eigvalsh(A)[-1]
    v0 = rand_field(L, Ls, 10)
    # the top of this tiny spectrum is nearly degenerate (gap ~1e-3), so the
    # Rayleigh quotient creeps up from below
    est = krylov.power_max(lambda v: dwf.mdagm(U, v, M5, 0.05), v0, 3000)
    assert est <= lmax * (1 + 1e-12)
    assert abs(est - lmax) / lmax < 2e-5
