"""Pins of the FP64 oracle's Chebyshev, coarsening, multigrid and force parts
(Secs. 3.1-3.4 of arXiv:2103.05034, and the HMC force derived from Sec. 6's
action) against closed forms, dense linear algebra, identities, finite
differences and the paper's printed counts (tests/golden/paper_counts.json)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import cheby, coarse, dwf, force, krylov, mg

M5 = 1.8
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))


# ------------------------------------------------------------ Chebyshev scalars
def test_chebyshev_recurrence_matches_trig_forms():
    x = np.linspace(-1, 1, 101)
    for n in (0, 1, 2, 7, 60):
        assert np.allclose(cheby.cheb_T(n, x), np.cos(n * np.arccos(x)), atol=1e-12)
    xo = np.array([1.01, 1.5, 3.0, -1.2])
    for n in (3, 12, 40):
        want = np.sign(xo) ** n * np.cosh(n * np.arccosh(np.abs(xo)))
        assert np.allclose(cheby.cheb_T(n, xo), want, rtol=1e-10)


def test_smoother_coeff_last_vanishes_and_interpolates():
    for a, b, N in [(0.5, 60.0, 12), (0.1, 10.0, 7)]:
        c = cheby.smoother_coeffs(a, b, N)
        assert abs(c[N]) < 1e-14 * np.max(np.abs(c))
        k = np.arange(N)
        nodes = a + (b - a) * (np.cos(np.pi * (k + 0.5) / N) + 1) / 2
        assert np.allclose(cheby.smoother_scalar(nodes, a, b, N), 1.0 / nodes, rtol=1e-12)


def test_filter_gain_matches_paper_order_of_magnitude():
    g = GOLD["filter_gain"]
    x0 = 2 * (0.0 - g["lambda_lo"]) / (g["lambda_max"] - g["lambda_lo"]) - 1
    gain = abs(cheby.cheb_T(g["m"], np.array([x0]))[0])
    assert np.log10(gain) == pytest.approx(np.log10(g["gain_order_of_magnitude"]), abs=0.5)


# ------------------------------------------------------------ operator level, dense tiny system
@pytest.fixture(scope="module")
def tiny():
    L = (2, 2, 2, 2)
    Ls = 4
    mf = 0.05
    U = synth.random_gauge(L, 0.7, 31)
    shape = (2, 2, 2, 2, Ls, 4, 3)
    n = int(np.prod(shape))
    D = np.zeros((n, n), complex)
    G = np.zeros((n, n), complex)
    for i in range(n):
        e = np.zeros(n, complex)
        e[i] = 1
        D[:, i] = dwf.ddw(U, e.reshape(shape), M5, mf).ravel()
        G[:, i] = dwf.gamma5_r5(e.reshape(shape)).ravel()
    return L, Ls, mf, U, shape, D, G


def test_filter_and_smoother_vs_eigendecomposition(tiny):
    L, Ls, mf, U, shape, D, G = tiny
    A = D.conj().T @ D
    lam, V = np.linalg.eigh(A)
    v = synth.gaussian_spinor(L, Ls, 3)
    appA = lambda w: dwf.mdagm(U, w, M5, mf)
    lo, hi, order = 0.3, 70.0, 9
    got = cheby.cheby_filter(appA, v, order, lo, hi).ravel()
    xl = 2 * (lam - lo) / (hi - lo) - 1
    want = V @ (cheby.cheb_T(order, xl) * (V.conj().T @ v.ravel()))
    assert np.allclose(got, want, rtol=1e-10, atol=1e-10)
    # smoother: p(M^dag M) M^dag with M = H (hermitian)
    H = G @ D
    appH = lambda w: dwf.hdw(U, w, M5, mf)
    z, nA = cheby.smoother_apply(appH, appH, v, 0.5, 60.0, 12)
    assert nA == 23
    lamH, VH = np.linalg.eigh(H)
    want = VH @ (cheby.smoother_scalar(lamH ** 2, 0.5, 60.0, 12) * lamH * (VH.conj().T @ v.ravel()))
    assert np.allclose(z.ravel(), want, rtol=1e-10, atol=1e-10)


def test_recursive_basis_vs_eigendecomposition_and_cost(tiny):
    L, Ls, mf, U, shape, D, G = tiny
    A = D.conj().T @ D
    lam, V = np.linalg.eigh(A)
    eta = synth.gaussian_spinor(L, Ls, 4)
    calls = [0]

    def appA(w):
        calls[0] += 1
        return dwf.mdagm(U, w, M5, mf)

    m, delta, nvec, lo, lmax = 7, 3, 4, 0.2, 70.0
    vecs = cheby.recursive_basis(appA, eta, m, delta, nvec, lo, lmax)
    assert calls[0] == m + (nvec - 1) * delta
    pre = cheby.cheb_T(m, 2 * (lam - lo) / (lmax - lo) - 1)
    c0 = V.conj().T @ eta.ravel()
    for k, phi in enumerate(vecs):
        f = pre * cheby.cheb_T(k * delta, 2 * lam / lmax - 1)
        want = V @ (f * c0)
        want /= np.linalg.norm(want)
        assert np.allclose(phi.ravel(), want, atol=1e-10)


def test_recursive_cost_model_matches_paper():
    """Cost m + (n-1) Delta of the recursive filter against the paper's counts and timings."""
    g = GOLD["recursive_cost"]
    assert (g["nvec"] - 1) * g["delta"] == g["further_multiplies"]
    s = GOLD["setup_time_ratio"]
    cost = lambda n: s["m"] + (n - 1) * s["delta"]
    model = cost(s["A_filtered"]) / cost(s["B_filtered"])
    assert model == pytest.approx(s["A_seconds"] / s["B_seconds"], abs=0.02)


def test_rbcg_count_convention_matches_paper():
    g = GOLD["rbcg_matmuls"]
    for it, mm in zip(g["iterations"], g["full_matmuls"]):
        assert 4 * it / 2 == mm  # four half-lattice hops = two full matmuls
    h = GOLD["hdcr_outer"]
    assert all(mm == 48 * o for o, mm in zip(h["outer"], h["fine_matmuls"]))


# ------------------------------------------------------------ coarsening
def make_basis(U, L, Ls, block, nvec, seed, mf):
    """Chirality-projected, block-orthonormalised basis from lightly filtered noise."""
    appA = lambda w: dwf.mdagm(U, w, M5, mf)
    raw = [cheby.cheby_filter(appA, synth.gaussian_spinor(L, Ls, seed + i), 4, 0.5, 70.0)
           for i in range(nvec)]
    half = nvec // 2
    vecs = [coarse.chiral_project(v, +1) for v in raw[:half]] + \
           [coarse.chiral_project(v, -1) for v in raw[half:]]
    return coarse.block_orthonormalise(vecs, block, [list(range(half)), list(range(half, nvec))])


@pytest.fixture(scope="module", params=[((4, 4, 4, 4), (2, 2, 2, 2)), ((4, 4, 2, 8), (2, 2, 2, 2))])
def coarse_case(request):
    L, block = request.param
    Ls = 4
    mf = 0.1
    U = synth.random_gauge(L, 0.5, 41)
    basis = make_basis(U, L, Ls, block, 4, 100, mf)
    return L, Ls, block, mf, U, basis


def test_block_orthonormal_and_chiral(coarse_case):
    L, Ls, block, mf, U, basis = coarse_case
    nb = len(basis)
    for j in range(nb):
        for k in range(nb):
            ip = coarse.block_inner(basis[j], basis[k], block)
            assert np.allclose(ip, 1.0 if j == k else 0.0, atol=1e-13)
    for k, phi in enumerate(basis):
        sgn = 1 if k < nb // 2 else -1
        assert np.allclose(dwf.gamma5_r5(phi), sgn * phi, atol=1e-14)


def test_coarse_stencil_equals_bruteforce(coarse_case):
    L, Ls, block, mf, U, basis = coarse_case
    A = coarse.coarse_build(U, basis, block, M5, mf)
    dense_stencil = coarse.coarse_dense_from_stencil(A)
    dense_bf = coarse.coarse_dense_bruteforce(U, basis, block, M5, mf)
    assert np.allclose(dense_stencil, dense_bf, atol=1e-12)
    # coarse operator of a hermitian H is hermitian; stencil form of it
    assert np.allclose(dense_bf, dense_bf.conj().T, atol=1e-12)
    assert np.allclose(A[0], np.conj(np.swapaxes(A[0], -1, -2)), atol=1e-12)
    for mu in range(4):
        ax = (3, 2, 1, 0)[mu]
        fwd = A[1 + 2 * mu]
        bwd_next = np.roll(A[2 + 2 * mu], -1, axis=ax)
        assert np.allclose(fwd, np.conj(np.swapaxes(bwd_next, -1, -2)), atol=1e-12)


def test_coarse_inherits_gamma5_hermiticity(coarse_case):
    """D_c = Gamma_5c A satisfies Gamma_5c D_c Gamma_5c = D_c^dag (Sec. 3.4)."""
    L, Ls, block, mf, U, basis = coarse_case
    dense = coarse.coarse_dense_bruteforce(U, basis, block, M5, mf)
    nb = len(basis)
    nc = dense.shape[0] // nb
    g5c = np.kron(np.eye(nc), np.diag([1.0] * (nb // 2) + [-1.0] * (nb // 2)))
    Dc = g5c @ dense
    assert np.allclose(g5c @ Dc @ g5c, Dc.conj().T, atol=1e-12)
    # and the restriction commutes with Gamma_5: P^dag Gamma_5 psi = Gamma_5c P^dag psi
    psi = synth.gaussian_spinor(L, Ls, 77)
    lhs = coarse.restrict(basis, dwf.gamma5_r5(psi), block)
    rhs = coarse.restrict(basis, psi, block) * np.array([1.0] * (nb // 2) + [-1.0] * (nb // 2))
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_coarse_apply_and_cgnr(coarse_case):
    L, Ls, block, mf, U, basis = coarse_case
    A = coarse.coarse_build(U, basis, block, M5, mf)
    dense = coarse.coarse_dense_bruteforce(U, basis, block, M5, mf)
    shp = A.shape[1:5] + (len(basis),)
    v = synth.complex_gaussian(5, shp)
    assert np.allclose(coarse.coarse_apply(A, v).ravel(), dense @ v.ravel(), atol=1e-12)
    e, it = coarse.coarse_cgnr(A, v, 1e-12, 2000)
    assert np.allclose(dense @ e.ravel(), v.ravel(), atol=1e-9 * np.linalg.norm(v))


def test_coarse_red_black_solve(coarse_case):
    """The red-black coarse solve (Sec. 5.3) reaches the dense solution, its
    Schur complement of the dense operator is hermitian, and it needs no
    more iterations than CG on A^2 for the same tolerance; odd coarse
    extents are refused."""
    L, Ls, block, mf, U, basis = coarse_case
    A = coarse.coarse_build(U, basis, block, M5, mf)
    shp = A.shape[1:5] + (len(basis),)
    v = synth.complex_gaussian(6, shp)
    if any(n % 2 for n in A.shape[1:5]):
        with pytest.raises(ValueError):
            coarse.coarse_rb_solve(A, v, 1e-12, 2000)
        return
    dense = coarse.coarse_dense_from_stencil(A)
    e, it = coarse.coarse_rb_solve(A, v, 1e-12, 2000)
    assert np.allclose(dense @ e.ravel(), v.ravel(), atol=1e-9 * np.linalg.norm(v))
    # Schur complement against the dense blocks
    nb = len(basis)
    par = np.repeat(coarse.coarse_parity_mask(A.shape[1:5]).ravel(), nb) > 0.5
    ie, io = np.where(par)[0], np.where(~par)[0]
    S = dense[np.ix_(ie, ie)] - dense[np.ix_(ie, io)] @ np.linalg.solve(dense[np.ix_(io, io)], dense[np.ix_(io, ie)])
    assert np.allclose(S, S.conj().T, atol=1e-10)
    _, it_full = coarse.coarse_cgnr(A, v, 1e-8, 2000)
    _, it_rb = coarse.coarse_rb_solve(A, v, 1e-8, 2000)
    assert it_rb <= it_full  # half the unknowns, no worse conditioned


def test_coarse_deflation(coarse_case):
    """Chebyshev-preconditioned Lanczos on the coarse A^2 finds its lowest
    eigenvalues (against a dense eigensolver), and the deflated coarse CG
    reaches the dense solution in fewer iterations than without deflation."""
    L, Ls, block, mf, U, basis = coarse_case
    A = coarse.coarse_build(U, basis, block, M5, mf)
    shp = A.shape[1:5] + (len(basis),)
    dense = coarse.coarse_dense_from_stencil(A)
    ev = np.linalg.eigvalsh(dense.conj().T @ dense)
    nev = 6
    AA = lambda u: coarse.coarse_apply(A, coarse.coarse_apply(A, u))
    lam_max = 1.1 * krylov.power_max(AA, synth.complex_gaussian(7, shp), 200)
    lam_lo = 0.5 * (ev[nev] + ev[nev + 1])
    theta, V = coarse.cheby_lanczos(AA, synth.complex_gaussian(8, shp), nev, 3 * nev, 8, lam_lo, lam_max)
    assert np.allclose(np.sort(theta), ev[:nev], rtol=1e-8, atol=1e-12 * ev[-1])
    for th, v in zip(theta, V):
        assert np.linalg.norm(AA(v) - th * v) <= 1e-6 * ev[-1] * np.linalg.norm(v)
    r = synth.complex_gaussian(9, shp)
    e, it_d = coarse.coarse_deflated_cgnr(A, r, theta, V, 1e-10, 5000)
    assert np.allclose(dense @ e.ravel(), r.ravel(), atol=1e-7 * np.linalg.norm(r))
    _, it_0 = coarse.coarse_cgnr(A, r, 1e-10, 5000)
    assert it_d < it_0


# ------------------------------------------------------------ V(1,1) and the MG solve
def test_vcycle_identity_dense(tiny):
    """The sequential x1, x2, x3 update (Eqs. 26-28) equals Eq. (31)'s
    [S(1 - MQ) + Q + (1 - QM)S + S(MQM - M)S] r0.  Eq. (32) rewrites the last
    term as + S P_L M S, but S(MQM - M)S = - S P_L M S: the sign is read from
    Eq. (31), which follows from the sequence."""
    L, Ls, mf, U, shape, D, G = tiny
    H = G @ D
    block = (2, 2, 2, 2)
    basis = make_basis(U, L, Ls, block, 4, 500, mf)
    A = coarse.coarse_build(U, basis, block, M5, mf)
    n = H.shape[0]
    P = np.stack([phi.ravel() for phi in basis], axis=1)  # one coarse site
    Ac = P.conj().T @ H @ P
    Q = P @ np.linalg.solve(Ac, P.conj().T)
    appH = lambda w: dwf.hdw(U, w, M5, mf)
    S = np.zeros((n, n), complex)
    for i in range(n):
        e = np.zeros(n, complex)
        e[i] = 1
        S[:, i] = cheby.smoother_apply(appH, appH, e.reshape(shape), 0.5, 60.0, 5)[0].ravel()
    I = np.eye(n)
    PL, PR = I - H @ Q, I - Q @ H
    K = S @ (I - H @ Q) + Q + (I - Q @ H) @ S + S @ (H @ Q @ H - H) @ S
    assert np.allclose(K, S @ PL + Q + PR @ S - S @ PL @ H @ S, atol=1e-10)
    r0 = synth.gaussian_spinor(L, Ls, 8)
    cnt = mg.MGCounter()
    got = mg.vcycle(appH, r0, basis, A, block, (0.5, 60.0, 5), 1e-14, 5000, cnt)
    assert np.allclose(got.ravel(), K @ r0.ravel(), rtol=1e-8, atol=1e-8 * np.linalg.norm(r0))
    assert cnt.fine == 2 * 9 + 2


def test_mg_solve_converges_to_dense_solution():
    L = (4, 4, 4, 4)
    Ls = 4
    mf = 0.05
    block = (2, 2, 2, 2)
    U = synth.random_gauge(L, 0.5, 51)
    basis = make_basis(U, L, Ls, block, 8, 600, mf)
    A = coarse.coarse_build(U, basis, block, M5, mf)
    b = synth.gaussian_spinor(L, Ls, 9)
    x, it, hist, cnt = mg.mg_solve(U, b, basis, A, block, M5, mf, 1e-10,
                                   smooth=(0.5, 60.0, 6), coarse_tol=0.02)
    assert krylov.true_residual(U, x, b, M5, mf) <= 1e-10
    xr, _, _ = krylov.rbcg_solve(U, b, M5, mf, 1e-13)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-7


# ------------------------------------------------------------ force
@pytest.fixture(scope="module")
def force_case():
    L = (4, 4, 4, 4)
    Ls = 4
    U = synth.random_gauge(L, 0.5, 61)
    masses = [0.05, 0.3]
    phis = [dwf.project_parity(synth.gaussian_spinor(L, Ls, 70 + i), L, 0) for i in range(2)]
    G = force.force(U, phis, masses, M5)
    return L, Ls, U, masses, phis, G


def test_force_is_traceless_antihermitian(force_case):
    L, Ls, U, masses, phis, G = force_case
    assert np.allclose(G, -dwf.dagger(G), atol=1e-14)
    assert np.allclose(np.trace(G, axis1=-2, axis2=-1), 0, atol=1e-13)


@pytest.mark.parametrize("kind", ["global", "single_link"])
def test_force_matches_finite_difference(force_case, kind):
    L, Ls, U, masses, phis, G = force_case
    if kind == "global":
        Q = synth.random_su3_algebra(U.shape[:-2], 81)
    else:
        Q = np.zeros_like(U)
        Q[1, 2, 3, 0, 2] = synth.random_su3_algebra((1,), 82)[0]
    fd = force.finite_difference(U, phis, masses, M5, Q, 1e-5)
    an = np.sum(np.trace(np.conj(np.swapaxes(G, -1, -2)) @ Q, axis1=-2, axis2=-1)).real
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3)


def test_force_gauge_covariance(force_case):
    L, Ls, U, masses, phis, G = force_case
    g = synth.random_gauge_transform(L, 91)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ dwf.dagger(dwf.shift(g, mu, +1))
    phig = [dwf.apply_color(g, p) for p in phis]
    Gg = force.force(Ug, phig, masses, M5)
    want = np.einsum("tzyxab,tzyxmbc,tzyxdc->tzyxmad", g, G, g.conj())
    assert np.allclose(Gg, want, atol=1e-10)


# ------------------------------------------------------------ Hasenbusch ratio
@pytest.fixture(scope="module")
def ratio_case():
    L = (4, 4, 4, 4)
    Ls = 4
    U = synth.random_gauge(L, 0.5, 63)
    phi = dwf.project_parity(synth.gaussian_spinor(L, Ls, 72), L, 0)
    return L, Ls, U, phi


def test_ratio_force_matches_finite_difference(ratio_case):
    """dS_r/deps along a random su(3) field against sum Re tr(G_r^dag Q)."""
    L, Ls, U, phi = ratio_case
    m1, m2 = 0.05, 0.3
    G = force.ratio_force(U, phi, m1, m2, M5)
    assert np.allclose(G, -dwf.dagger(G), atol=1e-14)
    Q = synth.random_su3_algebra(U.shape[:-2], 84)
    eps = 1e-5
    Up = np.einsum("...ij,...jk->...ik", force.exp_su3(eps * Q), U)
    Um = np.einsum("...ij,...jk->...ik", force.exp_su3(-eps * Q), U)
    fd = (force.ratio_action(Up, phi, m1, m2, M5) - force.ratio_action(Um, phi, m1, m2, M5)) / (2 * eps)
    an = np.sum(np.trace(np.conj(np.swapaxes(G, -1, -2)) @ Q, axis1=-2, axis2=-1)).real
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3)


def test_ratio_with_equal_masses_is_gauge_independent(ratio_case):
    """m1 = m2: S_r = phi^dag phi for every U, so its force vanishes while
    each of its two terms alone does not."""
    L, Ls, U, phi = ratio_case
    m = 0.1
    assert force.ratio_action(U, phi, m, m, M5) == pytest.approx(dwf.norm2(phi), rel=1e-11)
    G = force.ratio_force(U, phi, m, m, M5)
    G1 = force.force(U, [dwf.mpc_dag(U, phi, M5, m)], [m], M5)
    assert np.max(np.abs(G)) <= 1e-10 * np.max(np.abs(G1))
    assert np.max(np.abs(G1)) > 1e-3


def test_ratio_force_gauge_covariance(ratio_case):
    L, Ls, U, phi = ratio_case
    g = synth.random_gauge_transform(L, 93)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ dwf.dagger(dwf.shift(g, mu, +1))
    G = force.ratio_force(U, phi, 0.05, 0.3, M5)
    Gg = force.ratio_force(Ug, dwf.apply_color(g, phi), 0.05, 0.3, M5)
    want = np.einsum("tzyxab,tzyxmbc,tzyxdc->tzyxmad", g, G, g.conj())
    assert np.allclose(Gg, want, atol=1e-10)
