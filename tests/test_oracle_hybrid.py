"""Pins of the FP64 oracle of the hybrid three-level multigrid (Algorithm F of
arXiv:2103.05034, Sec. 4) against closed forms, dense linear algebra, exact
solves with complete bases and the paper's printed counts."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import coarse, dwf, hybrid, krylov

M5 = 1.8
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))


def gauss4(L, seed):
    """A complex Gaussian 4D spinor field (T,Z,Y,X,4,3)."""
    return synth.complex_gaussian(seed, (L[3], L[2], L[1], L[0], 4, 3))


def unit_gauge(L):
    U = np.zeros((L[3], L[2], L[1], L[0], 4, 3, 3), complex)
    U[...] = np.eye(3)
    return U


# ------------------------------------------------------------ Eq. (1) in 4D
def test_wilson_free_field_plane_wave():
    """Free field: D_W(m) e^{ipx} chi = (m + sum_mu (1 - cos p_mu) + i sum_mu gamma_mu sin p_mu) e^{ipx} chi."""
    L = (4, 4, 2, 6)
    U = unit_gauge(L)
    n = (1, 3, 1, 2)
    p = [2 * np.pi * n[m] / L[m] for m in range(4)]
    t, z, y, x = np.meshgrid(np.arange(L[3]), np.arange(L[2]), np.arange(L[1]), np.arange(L[0]), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    chi = synth.complex_gaussian(5, (4, 3))
    psi = phase[..., None, None] * chi
    for m in (-0.95, 0.3):
        M = (m + sum(1 - np.cos(pm) for pm in p)) * np.eye(4) + 1j * sum(dwf.GAMMA[mu] * np.sin(p[mu]) for mu in range(4))
        want = phase[..., None, None] * (M @ chi)
        assert np.allclose(hybrid.wilson(U, psi, m), want, atol=1e-13)


def test_wilson_adjoint_and_gamma5_hermiticity():
    L = (4, 4, 4, 4)
    U = synth.random_gauge(L, 0.5, 61)
    u, v = gauss4(L, 1), gauss4(L, 2)
    m = -0.95
    assert np.isclose(dwf.inner(u, hybrid.wilson(U, v, m)), dwf.inner(hybrid.wilson(U, u, m, dag=True), v), rtol=1e-12)
    g5 = lambda w: dwf.apply_spin(dwf.GAMMA5, w)
    assert np.allclose(g5(hybrid.wilson(U, g5(v), m)), hybrid.wilson(U, v, m, dag=True), atol=1e-12)


# ------------------------------------------------------------ first coarsening (4D D_W)
@pytest.fixture(scope="module", params=[((4, 4, 4, 4), (2, 2, 2, 2)), ((4, 4, 2, 8), (2, 2, 2, 2))])
def case4(request):
    L, block = request.param
    U = synth.random_gauge(L, 0.5, 71)
    etas = [gauss4(L, 200 + i) for i in range(4)]
    b4 = hybrid.basis4(U, etas, -0.95, 1.0, 60.0, 3, block)
    return L, block, U, b4


def test_basis4_orthonormal_and_chiral(case4):
    L, block, U, b4 = case4
    nb = len(b4)
    for j in range(nb):
        for k in range(nb):
            assert np.allclose(coarse.block_inner(b4[j], b4[k], block), 1.0 if j == k else 0.0, atol=1e-13)
    for k, phi in enumerate(b4):
        sgn = 1 if k < nb // 2 else -1
        assert np.allclose(dwf.apply_spin(dwf.GAMMA5, phi), sgn * phi, atol=1e-14)


def test_coarse_build4_equals_bruteforce(case4):
    """The 9-point stencil of -1/2 D_hop on the 4D block basis equals the dense
    P4^dag (-1/2 D_hop) P4, formed by hopping every block basis vector."""
    L, block, U, b4 = case4
    B = hybrid.coarse_build4(U, b4, block)
    Lc = coarse.coarse_dims(L, block)
    nc, nb = int(np.prod(Lc)), len(b4)
    D = np.zeros((nc * nb, nc * nb), complex)
    for c in range(nc):
        sel = np.zeros(nc)
        sel[c] = 1.0
        sel = sel.reshape(Lc[3], Lc[2], Lc[1], Lc[0])
        for k, phi in enumerate(b4):
            col = -0.5 * dwf.dhop(U, (coarse._expand(sel, block, phi.shape) * phi)[:, :, :, :, None])[:, :, :, :, 0]
            D[:, c * nb + k] = np.stack([coarse.block_inner(pj, col, block) for pj in b4], axis=-1).ravel()
    assert np.allclose(coarse.coarse_dense_from_stencil(B), D, atol=1e-12)


# ------------------------------------------------------------ level 1: the coarse domain wall operator
@pytest.fixture(scope="module")
def case1():
    L, block, Ls, mf = (4, 4, 4, 4), (2, 2, 2, 2), 4, 0.05
    U = synth.random_gauge(L, 0.5, 81)
    b4 = hybrid.basis4(U, [gauss4(L, 300 + i) for i in range(4)], -0.95, 1.0, 60.0, 3, block)
    B = hybrid.coarse_build4(U, b4, block)
    return L, block, Ls, mf, U, b4, B


def dense_of(apply, shape):
    n = int(np.prod(shape))
    D = np.zeros((n, n), complex)
    for i in range(n):
        e = np.zeros(n, complex)
        e[i] = 1
        D[:, i] = apply(e.reshape(shape)).ravel()
    return D


def test_level1_operator_equals_projected_ddw(case1):
    """M_1 (fifth-dimension matrix by chirality plus the coarse hop on every s)
    equals P1^dag D_DW P1 built by prolonging, applying the fine D_DW and
    restricting; the basis is orthonormal so P1^dag P1 = 1."""
    L, block, Ls, mf, U, b4, B = case1
    Lc = coarse.coarse_dims(L, block)
    shape = (Lc[3], Lc[2], Lc[1], Lc[0], len(b4), Ls)
    M1 = dense_of(lambda v: hybrid.level1_apply(B, v, M5, mf, 2), shape)
    Pb = dense_of(lambda v: hybrid.restrict1(b4, dwf.ddw(U, hybrid.prolong1(b4, v, block), M5, mf), block), shape)
    assert np.allclose(M1, Pb, atol=1e-12)
    PP = dense_of(lambda v: hybrid.restrict1(b4, hybrid.prolong1(b4, v, block), block), shape)
    assert np.allclose(PP, np.eye(PP.shape[0]), atol=1e-13)
    # H_1 = Gamma5_1 M_1 is hermitian (inherited Gamma_5 hermiticity) and equals P1^dag H_DW P1
    H1 = dense_of(lambda v: hybrid.level1_herm(B, v, M5, mf, 2), shape)
    assert np.allclose(H1, H1.conj().T, atol=1e-12)
    PH = dense_of(lambda v: hybrid.restrict1(b4, dwf.hdw(U, hybrid.prolong1(b4, v, block), M5, mf), block), shape)
    assert np.allclose(H1, PH, atol=1e-12)


@pytest.fixture(scope="module")
def case2(case1):
    L, block, Ls, mf, U, b4, B = case1
    Lc = coarse.coarse_dims(L, block)
    shape = (Lc[3], Lc[2], Lc[1], Lc[0], len(b4), Ls)
    etas = [synth.complex_gaussian(400 + i, shape) for i in range(4)]
    b2 = hybrid.basis2(B, etas, M5, mf, 2, 0.5, 60.0, 3)
    return shape, b2


def test_basis2_orthonormal_and_chiral(case1, case2):
    shape, b2 = case2
    nb = len(b2)
    for i in range(nb):
        for j in range(nb):
            assert np.allclose(coarse.block_inner(b2[i], b2[j], hybrid.SITE), 1.0 if i == j else 0.0, atol=1e-13)
    for i, phi in enumerate(b2):
        sgn = 1 if i < nb // 2 else -1
        assert np.allclose(hybrid.gamma5_1(phi, 2), sgn * phi, atol=1e-14)


def test_coarse_build2_equals_bruteforce(case1, case2):
    """The level-2 stencil equals the dense P2^dag H_1 P2."""
    L, block, Ls, mf, U, b4, B = case1
    shape, b2 = case2
    A2 = hybrid.coarse_build2(B, b2, M5, mf, 2)
    H1 = dense_of(lambda v: hybrid.level1_herm(B, v, M5, mf, 2), shape)
    n2 = int(np.prod(shape[:4])) * len(b2)
    P2 = np.stack([hybrid.prolong2(b2, e.reshape(shape[:4] + (len(b2),))).ravel() for e in np.eye(n2)], axis=1)
    assert np.allclose(coarse.coarse_dense_from_stencil(A2), P2.conj().T @ H1 @ P2, atol=1e-12)
    # the restriction is P2^dag
    v = synth.complex_gaussian(9, shape)
    assert np.allclose(hybrid.restrict2(b2, v).ravel(), P2.conj().T @ v.ravel(), atol=1e-12)


# ------------------------------------------------------------ the solve
def test_complete_bases_give_the_exact_solve_in_one_step():
    """With complete bases at both levels (P1, P2 unitary) and an exact
    coarse-coarse solve, the coarse correction alone inverts H_DW: one outer
    iteration reaches the coarse solver's precision."""
    L, Ls, mf, block = (2, 2, 2, 2), 2, 0.1, (1, 1, 1, 1)
    U = synth.random_gauge(L, 0.5, 91)
    b4 = hybrid.basis4(U, [gauss4(L, 500 + i) for i in range(12)], -0.5, 1.0, 60.0, 1, block)
    B = hybrid.coarse_build4(U, b4, block)
    shape = (L[3], L[2], L[1], L[0], 12, Ls)
    b2 = hybrid.basis2(B, [synth.complex_gaussian(600 + i, shape) for i in range(24)], M5, mf, 6, 0.5, 60.0, 1)
    A2 = hybrid.coarse_build2(B, b2, M5, mf, 6)
    h = hybrid.Hybrid(U, M5, mf, block, b4, B, b2, A2, smooth=(0.5, 60.0, 3), smooth1=(0.5, 60.0, 0), kcycle=1,
                      coarse_tol=1e-14, coarse_maxiter=5000)
    b = synth.gaussian_spinor(L, Ls, 7)
    x, it, hist, cnt = hybrid.hybrid_solve(h, b, 1e-9)
    assert it == 1
    assert krylov.true_residual(U, x, b, M5, mf) <= 1e-9


@pytest.mark.parametrize("smooth1,kcycle", [((0.5, 60.0, 0), 1), ((0.5, 60.0, 3), 2)])
def test_hybrid_solve_converges_to_dense_solution(smooth1, kcycle):
    L, Ls, mf, block = (4, 4, 4, 4), 4, 0.05, (2, 2, 2, 2)
    U = synth.random_gauge(L, 0.5, 101)
    b4 = hybrid.basis4(U, [gauss4(L, 700 + i) for i in range(8)], -0.95, 1.0, 60.0, 6, block)
    B = hybrid.coarse_build4(U, b4, block)
    shape = (2, 2, 2, 2, 8, Ls)
    b2 = hybrid.basis2(B, [synth.complex_gaussian(800 + i, shape) for i in range(8)], M5, mf, 4, 0.5, 60.0, 6)
    A2 = hybrid.coarse_build2(B, b2, M5, mf, 4)
    h = hybrid.Hybrid(U, M5, mf, block, b4, B, b2, A2, smooth=(0.5, 60.0, 6), smooth1=smooth1, kcycle=kcycle,
                      coarse_tol=0.02)
    b = synth.gaussian_spinor(L, Ls, 11)
    x, it, hist, cnt = hybrid.hybrid_solve(h, b, 1e-8)
    assert krylov.true_residual(U, x, b, M5, mf) <= 1e-8
    xr, _, _ = krylov.rbcg_solve(U, b, M5, mf, 1e-13)
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) < 1e-6
    # the W-cycle: kcycle coarse-coarse solves per fine outer iteration
    assert cnt.solves2 == kcycle * it


def test_paper_counts_for_algorithm_f():
    """Table 9: Algorithm F's fine matrix multiplies are 48 per outer
    iteration (the count of HDCR's Table 7), with two coarse-coarse solves per
    outer iteration; the composite blocking is 2^4 x 16."""
    g = GOLD["hybrid_outer"]
    assert g["fine_matmuls"] == 48 * g["outer"]
    assert g["coarse_coarse_solves_per_outer"] == 2
    comp = [a * b for a, b in zip(g["block1"], g["block2"])]
    assert comp == [2, 2, 2, 2, 16]


def test_degenerate_wcycle_is_rejected():
    """Without a level-1 smoother the preconditioner K = P2 A_2^-1 P2^dag
    satisfies K H_1 K = K: a second GCR step would add nothing (the setup
    rejects kcycle > 1 then).  Checked on the dense level-1 operator."""
    L, Ls, mf, block = (4, 4, 4, 4), 4, 0.3, (2, 2, 2, 2)
    U = synth.random_gauge(L, 0.5, 111)
    b4 = hybrid.basis4(U, [gauss4(L, 900 + i) for i in range(4)], -0.95, 1.0, 60.0, 3, block)
    B = hybrid.coarse_build4(U, b4, block)
    shape = (2, 2, 2, 2, 4, Ls)
    b2 = hybrid.basis2(B, [synth.complex_gaussian(950 + i, shape) for i in range(8)], M5, mf, 2, 0.5, 60.0, 3)
    A2 = hybrid.coarse_build2(B, b2, M5, mf, 2)
    H1 = dense_of(lambda v: hybrid.level1_herm(B, v, M5, mf, 2), shape)
    n2 = int(np.prod(shape[:4])) * len(b2)
    P2 = np.stack([hybrid.prolong2(b2, e.reshape(shape[:4] + (len(b2),))).ravel() for e in np.eye(n2)], axis=1)
    K = P2 @ np.linalg.solve(coarse.coarse_dense_from_stencil(A2), P2.conj().T)
    assert np.allclose(K @ H1 @ K, K, atol=1e-10)
    with pytest.raises(ValueError):
        hybrid.Hybrid(U, M5, mf, block, b4, B, b2, A2, smooth1=(0.5, 60.0, 0), kcycle=2)
