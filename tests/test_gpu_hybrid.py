"""GPU parity of the hybrid three-level multigrid (Algorithm F of
arXiv:2103.05034, Sec. 4) through the C ABI against the FP64 oracle
(oracle/hybrid.py).

Tolerances: parts computed in FP64 from the same inputs (the 4D stencil B,
the level-2 stencil from the exported level-2 basis) 1e-11 relative; FP32
filters and FP32 level operators 1e-5 (a few hundred FP32 roundings of O(1)
numbers, Chebyshev orders <= 8); iterative results as stated per test."""
import numpy as np
import pytest
import torch

import synth
from oracle import coarse, dwf, hybrid, krylov
from paper_2103_05034_gb300 import layout, ops
from paper_2103_05034_gb300._lib import COARSE_CG, COARSE_DEFLATED, COARSE_RB, F32, F64, DWFError

from gpu_helpers import dev_to_full_canon, full_dev, rel

pytestmark = pytest.mark.gpu
M5 = 1.8
DEV = "cuda"


def gauss4(L, seed):
    return synth.complex_gaussian(seed, (L[3], L[2], L[1], L[0], 4, 3))


def slices_dev(fields, L):
    """nv 4D fields as the slices of a full field with Ls = nv (FP64, device)."""
    st = np.stack(fields, axis=4)  # (T, Z, Y, X, nv, 4, 3)
    return torch.from_numpy(layout.complex_to_real(layout.to_full(st, L), F64)).to(DEV)


def slices_canon(t, L, nv):
    a = layout.real_to_complex(t.double().cpu().numpy()).reshape(2, -1, 4, 3, nv)
    full = layout.from_full(a, L)
    return [full[:, :, :, :, k] for k in range(nv)]


def l1_dev(vecs, prec=F32):
    """Level-1 vectors (Tc, Zc, Yc, Xc, nb4, Ls) -> device [nc1][nb4][Ls][nvec]."""
    return torch.from_numpy(layout.complex_to_real(np.stack(vecs, axis=-1), prec)).to(DEV)


def l1_canon(t, shape, nvec):
    a = layout.real_to_complex(t.double().cpu().numpy()).reshape(shape + (nvec,))
    return [a[..., v] for v in range(nvec)]


def stencil_canon(t, Lc, nb):
    """Device [nc][9][nb][nb] (FP64) -> oracle (9, Tc, Zc, Yc, Xc, nb, nb)."""
    a = layout.real_to_complex(t.double().cpu().numpy()).reshape(-1, 9, nb, nb)
    return np.ascontiguousarray(a.transpose(1, 0, 2, 3)).reshape((9, Lc[3], Lc[2], Lc[1], Lc[0], nb, nb))


class Case:
    """A hybrid setup on the GPU and the oracle's objects built from its
    exported bases (so that every later comparison starts from the same data)."""

    def __init__(self, L, Ls, mf, block, nb4, nb2, filter4, filter1, smooth1=(0.5, 60.0, 3), kcycle=2,
                 coarse_tol=0.02, coarse_solver=COARSE_CG, deflation=(0, 0, 0, 0.0), seed=0, mass4=-0.95,
                 maxiter=200):
        self.L, self.Ls, self.mf, self.block, self.nb4, self.nb2 = L, Ls, mf, block, nb4, nb2
        self.filter4, self.filter1, self.mass4 = filter4, filter1, mass4
        self.U = synth.random_gauge(L, 0.5, 1100 + seed)
        self.ctx = ops.Context(L, Ls, M5, self.U)
        self.Lc = tuple(L[m] // block[m] for m in range(4))
        self.shape1 = (self.Lc[3], self.Lc[2], self.Lc[1], self.Lc[0], nb4, Ls)
        self.eta4 = [gauss4(L, 1200 + seed * 100 + i) for i in range(nb4)]
        self.eta1 = [synth.complex_gaussian(1300 + seed * 100 + i, self.shape1) for i in range(nb2)]
        self.p = ops.mg_params(block, 0, mf, smooth=(0.5, 60.0, 6), coarse_tol=coarse_tol, coarse_maxiter=2000,
                               nkrylov=8, maxiter=maxiter, coarse_solver=coarse_solver, deflation=deflation)
        self.hp = ops.hybrid_params(block, nb4, nb2, mass4=mass4, filter4=filter4, filter1=filter1,
                                    smooth1=smooth1, kcycle=kcycle)
        self.smooth1, self.kcycle = smooth1, kcycle
        self.G = ops.HybridMG(self.ctx, self.p, self.hp, slices_dev(self.eta4, L), l1_dev(self.eta1, F64))
        self.b4 = slices_canon(self.G.export(0), L, nb4)
        self.B = stencil_canon(self.G.export(1), self.Lc, nb4)
        self.b2 = l1_canon(self.G.export(2), self.shape1, nb2)
        self.A2 = stencil_canon(self.G.export(3), self.Lc, nb2)

    def oracle(self, coarse_tol=0.02):
        return hybrid.Hybrid(self.U, M5, self.mf, self.block, self.b4, self.B, self.b2, self.A2,
                             smooth=(0.5, 60.0, 6), smooth1=self.smooth1, kcycle=self.kcycle, coarse_tol=coarse_tol,
                             coarse_maxiter=5000)

    def close(self):
        self.G.close()
        self.ctx.close()


@pytest.fixture(scope="module", params=[4, 16], ids=["nb4_4", "nb4_16"])
def case(request):
    c = Case((4, 4, 4, 4), 4, 0.05, (2, 2, 2, 2), request.param, 8, (1.0, 60.0, 6), (0.5, 60.0, 6))
    yield c
    c.close()


# ------------------------------------------------------------ the 4D coarsening
def test_basis4_matches_oracle(case):
    """FP32 filter of D_W^dag D_W, gamma_5 projection and FP64 block
    Cholesky-QR against the oracle's FP64 filter and MGS."""
    lo, hi, order = case.filter4
    want = hybrid.basis4(case.U, case.eta4, case.mass4, lo, hi, order, case.block)
    for g, w in zip(case.b4, want):
        assert rel(g, w) < 1e-5
    nb = case.nb4
    for j in range(nb):
        for k in range(nb):
            ip = coarse.block_inner(case.b4[j], case.b4[k], case.block)
            assert np.allclose(ip, 1.0 if j == k else 0.0, atol=1e-12)
    for k, phi in enumerate(case.b4):
        assert np.array_equal(dwf.apply_spin(dwf.GAMMA5, phi), (1 if k < nb // 2 else -1) * phi)


def test_stencil4_matches_oracle(case):
    """B = P4^dag (-1/2 D_hop) P4 built in FP64 on the GPU's basis."""
    want = hybrid.coarse_build4(case.U, case.b4, case.block)
    assert rel(case.B, want) < 1e-11


def test_level1_operators(case):
    """M_1, H_1 (FP32 stencil) on three level-1 vectors at once, and the
    restriction / prolongation of both levels, against the oracle."""
    G, shape = case.G, case.shape1
    vs = [synth.complex_gaussian(1400 + i, shape) for i in range(3)]
    vin = l1_dev(vs)
    out = torch.zeros_like(vin)
    for op, f in ((0, hybrid.level1_apply), (1, hybrid.level1_herm)):
        G.level1(op, out, vin, 3)
        got = l1_canon(out, shape, 3)
        for g, v in zip(got, vs):
            assert rel(g, f(case.B, v, M5, case.mf, case.nb4 // 2)) < 1e-5
    # P1^dag on two fine fields, P1 on two level-1 vectors
    L, Ls = case.L, case.Ls
    psis = [synth.gaussian_spinor(L, Ls, 1500 + i) for i in range(2)]
    fin = torch.cat([full_dev(p, L, F32).reshape(-1) for p in psis])
    r1 = torch.zeros(2 * 2 * case.G.n1, dtype=torch.float32, device=DEV)
    G.level1(2, r1, fin, 2)
    for g, p in zip(l1_canon(r1, shape, 2), psis):
        assert rel(g, hybrid.restrict1(case.b4, p, case.block)) < 1e-5
    fout = torch.zeros_like(fin)
    G.level1(3, fout, l1_dev(vs[:2]), 2)
    n = fin.numel() // 2
    for i in range(2):
        got = dev_to_full_canon(fout[i * n:(i + 1) * n], L, Ls)
        assert rel(got, hybrid.prolong1(case.b4, vs[i], case.block)) < 1e-5
    # P2^dag, P2
    v = vs[0]
    r2 = torch.zeros(2 * case.G.nc1 * case.nb2, dtype=torch.float32, device=DEV)
    G.level1(4, r2, l1_dev([v]), 1)
    want = hybrid.restrict2(case.b2, v)
    assert rel(layout.real_to_complex(r2.double().cpu().numpy()).reshape(want.shape), want) < 1e-5
    e2 = synth.complex_gaussian(1600, want.shape)
    o1 = torch.zeros(2 * case.G.n1, dtype=torch.float32, device=DEV)
    G.level1(5, o1, torch.from_numpy(layout.complex_to_real(e2, F32)).to(DEV), 1)
    assert rel(l1_canon(o1, shape, 1)[0], hybrid.prolong2(case.b2, e2)) < 1e-5


# ------------------------------------------------------------ the second coarsening
def test_basis2_and_stencil2_match_oracle(case):
    """Level-2 basis (FP32 filter of H_1^2, Gamma5_1 halves, per-site
    Cholesky-QR) against the oracle's FP64 filter and MGS on the GPU's B; the
    level-2 stencil (FP64 sums) against the oracle's on the GPU's basis."""
    lo, hi, order = case.filter1
    want = hybrid.basis2(case.B, case.eta1, M5, case.mf, case.nb4 // 2, lo, hi, order)
    for g, w in zip(case.b2, want):
        assert rel(g, w) < 1e-4
    nb = case.nb2
    for i in range(nb):
        for j in range(nb):
            ip = coarse.block_inner(case.b2[i], case.b2[j], hybrid.SITE)
            assert np.allclose(ip, 1.0 if i == j else 0.0, atol=2e-6)
    for i, phi in enumerate(case.b2):
        assert rel(hybrid.gamma5_1(phi, case.nb4 // 2), (1 if i < nb // 2 else -1) * phi) < 1e-6
    A2 = hybrid.coarse_build2(case.B, case.b2, M5, case.mf, case.nb4 // 2)
    assert rel(case.A2, A2) < 1e-11
    # inherited Gamma_5 hermiticity: A_+mu(x) = A_-mu(x+mu)^dag, A_0 hermitian
    A0 = case.A2[0]
    assert rel(A0, np.conj(np.swapaxes(A0, -1, -2))) < 1e-6


@pytest.mark.parametrize("smooth1,kcycle", [((0.5, 60.0, 0), 1), ((0.5, 60.0, 3), 2)],
                         ids=["nosmooth_k1", "smooth3_k2"])
def test_level1_wcycle_solve(case, smooth1, kcycle):
    """The level-1 GCR (each iteration a level-1 V(1,1) around a level-2 CG on
    A_2^2 to 1e-6) against the oracle's on the same bases and stencils: one
    iteration without the level-1 smoother, two with it (without a smoother a
    second iteration would only amplify rounding: K H_1 K = K).  FP32 coarse
    solves against FP64 ones; the heavier mass 0.3 keeps A_2 well
    conditioned so that they agree to about 1e-6."""
    c = Case(case.L, case.Ls, 0.3, case.block, case.nb4, case.nb2, case.filter4, case.filter1,
             smooth1=smooth1, kcycle=kcycle, coarse_tol=1e-6, seed=0)
    try:
        r = synth.complex_gaussian(1700, c.shape1)
        out = torch.zeros(2 * c.G.n1, dtype=torch.float32, device=DEV)
        c.G.level1(6, out, l1_dev([r]), 1)
        got = l1_canon(out, c.shape1, 1)[0]
        h = c.oracle(coarse_tol=1e-6)
        cnt = hybrid.Counter()
        want = hybrid.level1_solve(h, r, cnt)
        assert cnt.solves2 == kcycle
        assert rel(got, want) < 1e-3
        # two GCR steps reduce the level-1 residual
        assert np.linalg.norm(r - h.H1(got)) < np.linalg.norm(r)
    finally:
        c.close()


# ------------------------------------------------------------ the solve
def test_hybrid_solve_matches_oracle(case):
    """mg_solve over the hybrid levels reaches the FP64 true residual 1e-8;
    the solution matches the oracle's red-black CG solution, and the outer
    iteration count matches the oracle's Algorithm F solve on the same bases
    (FP32 inner arithmetic against FP64)."""
    L, Ls = case.L, case.Ls
    b = synth.gaussian_spinor(L, Ls, 1800)
    bd = full_dev(b, L, F64)
    xd = torch.zeros_like(bd)
    st = ops.mg_solve(case.G, xd, bd, 1e-8)
    x = dev_to_full_canon(xd, L, Ls)
    res = krylov.true_residual(case.U, x, b, M5, case.mf)
    assert res <= 1e-8 * 1.01, st
    xr, _, _ = krylov.rbcg_solve(case.U, b, M5, case.mf, 1e-13)
    assert rel(x, xr) < 1e-6
    xo, it_or, _, cnt = hybrid.hybrid_solve(case.oracle(), b, 1e-8)
    print(f"hybrid solve nb4={case.nb4}: {st['iterations']} outer (oracle {it_or}), "
          f"{st['coarse_iterations']} level-2 CG iterations (oracle {cnt.coarse})")
    assert abs(st["iterations"] - it_or) <= max(3, it_or // 5)
    assert st["coarse_iterations"] > 0 and st["graph_replays"] == 0


@pytest.mark.parametrize("solver", ["rb", "deflated"])
def test_hybrid_solve_level2_solvers(case, solver):
    """The level-2 solve by red-black CG or from the deflation guess: the
    hybrid solve still reaches 1e-8."""
    kw = dict(coarse_solver=COARSE_RB) if solver == "rb" else \
        dict(coarse_solver=COARSE_DEFLATED, deflation=(16, 48, 6, 0.05))
    c = Case(case.L, case.Ls, case.mf, case.block, case.nb4, case.nb2, case.filter4, case.filter1, seed=0, **kw)
    try:
        b = synth.gaussian_spinor(c.L, c.Ls, 1801)
        bd = full_dev(b, c.L, F64)
        xd = torch.zeros_like(bd)
        st = ops.mg_solve(c.G, xd, bd, 1e-8)
        print(f"hybrid solve at Ls 16, nb4 24, nb2 32: {st['iterations']} outer, "
              f"{st['coarse_iterations']} level-2 CG iterations")
        x = dev_to_full_canon(xd, c.L, c.Ls)
        assert krylov.true_residual(c.U, x, b, M5, c.mf) <= 1e-8 * 1.01, st
    finally:
        c.close()


def test_hybrid_rejects_bad_parameters():
    L, Ls = (4, 4, 4, 4), 4
    U = synth.random_gauge(L, 0.5, 7)
    ctx = ops.Context(L, Ls, M5, U)
    try:
        p = ops.mg_params((2, 2, 2, 2), 0, 0.05)
        eta4 = torch.zeros(2 * 2 * ctx.Vh * 12 * 8, dtype=torch.float64, device=DEV)
        eta1 = torch.zeros(2 * 16 * 8 * Ls * 8, dtype=torch.float64, device=DEV)
        for kw in (dict(nb4=6), dict(nb2=7), dict(nb2=66), dict(mass4=-4.5), dict(block=(3, 2, 2, 2)),
                   dict(smooth1=(0.5, 60.0, 0))):
            hp = ops.hybrid_params(kw.get("block", (2, 2, 2, 2)), kw.get("nb4", 8), kw.get("nb2", 8),
                                   mass4=kw.get("mass4", -0.95), smooth1=kw.get("smooth1", (0.5, 60.0, 4)))
            with pytest.raises(DWFError):
                ops.HybridMG(ctx, p, hp, eta4, eta1)
    finally:
        ctx.close()


def test_hybrid_at_benchmark_shapes():
    """The shapes of Algorithm F's table (Table 3) on a small lattice: 24 4D
    vectors (the Ls = 24 hopping kernels on the 4D basis), Ls = 16, 32
    level-2 vectors (the nb = 32 coarse CG); B and the level-2 stencil against
    the oracle on the GPU's bases, the level-1 operator on one vector, and a
    converged solve."""
    c = Case((8, 4, 4, 8), 16, 0.05, (2, 2, 2, 2), 24, 32, (1.0, 60.0, 12), (0.5, 60.0, 12), seed=3,
             maxiter=600)
    try:
        assert rel(c.B, hybrid.coarse_build4(c.U, c.b4, c.block)) < 1e-11
        assert rel(c.A2, hybrid.coarse_build2(c.B, c.b2, M5, c.mf, 12)) < 1e-11
        v = synth.complex_gaussian(1900, c.shape1)
        out = torch.zeros(2 * c.G.n1, dtype=torch.float32, device=DEV)
        c.G.level1(1, out, l1_dev([v]), 1)
        assert rel(l1_canon(out, c.shape1, 1)[0], hybrid.level1_herm(c.B, v, M5, c.mf, 12)) < 1e-5
        b = synth.gaussian_spinor(c.L, c.Ls, 1901)
        bd = full_dev(b, c.L, F64)
        xd = torch.zeros_like(bd)
        st = ops.mg_solve(c.G, xd, bd, 1e-8)
        print(f"hybrid solve at Ls 16, nb4 24, nb2 32: {st['iterations']} outer, "
              f"{st['coarse_iterations']} level-2 CG iterations")
        x = dev_to_full_canon(xd, c.L, c.Ls)
        assert krylov.true_residual(c.U, x, b, M5, c.mf) <= 1e-8 * 1.01, st
    finally:
        c.close()
