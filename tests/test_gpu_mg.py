"""GPU parity of the HDCR multigrid path through the C ABI against the FP64
oracle (Secs. 3.1-3.4 of arXiv:2103.05034).

Tolerances: FP64 kernels 1e-11 relative (norm-wise); FP32 kernels 1e-5
relative (a few hundred FP32 roundings of O(1) numbers, 6e-8 each, with
Chebyshev recurrences of order <= 12 amplifying by at most ~10); iterative
results are compared as stated per test."""
import numpy as np
import pytest
import torch

import synth
from oracle import cheby, coarse, dwf, krylov, mg
from paper_2103_05034_gb300 import layout, ops
from paper_2103_05034_gb300._lib import F32, F64, SUBSPACE_BATCH, SUBSPACE_RECURSIVE

from gpu_helpers import dev_to_full_canon, full_dev, rel

pytestmark = pytest.mark.gpu
M5 = 1.8


def fulls_dev(vecs, L, prec):
    return torch.cat([full_dev(v, L, prec).reshape(-1) for v in vecs])


def fulls_canon(t, L, Ls, n):
    a = layout.real_to_complex(t.double().cpu().numpy()).reshape(n, 2, -1, 4, 3, Ls)
    return [layout.from_full(a[i], L) for i in range(n)]


@pytest.fixture(scope="module")
def small():
    L, Ls, mf = (4, 4, 4, 4), 4, 0.05
    U = synth.random_gauge(L, 0.5, 41)
    ctx = ops.Context(L, Ls, M5, U)
    appA = lambda v: dwf.mdagm(U, v, M5, mf)
    lmax = krylov.power_max(appA, synth.gaussian_spinor(L, Ls, 1), 200) * 1.1
    yield L, Ls, mf, U, ctx, lmax
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(F64, 1e-11), (F32, 1e-5)])
def test_cheby_filter_batched(small, prec, tol):
    L, Ls, mf, U, ctx, lmax = small
    vs = [synth.gaussian_spinor(L, Ls, 50 + i) for i in range(3)]
    inp = fulls_dev(vs, L, prec)
    out = torch.zeros_like(inp)
    order, lo = 9, 0.5
    ops.cheby_filter(ctx, out, inp, 3, lo, lmax, order, mf)
    got = fulls_canon(out, L, Ls, 3)
    appA = lambda v: dwf.mdagm(U, v, M5, mf)
    for g, v in zip(got, vs):
        err = rel(g, cheby.cheby_filter(appA, v, order, lo, lmax))
        print(f"cheby_filter prec={prec} order={order}: rel err {err:.3e}")
        assert err < tol


@pytest.mark.parametrize("prec,tol", [(F64, 1e-10), (F32, 1e-5)])
def test_recursive_basis(small, prec, tol):
    L, Ls, mf, U, ctx, lmax = small
    eta = synth.gaussian_spinor(L, Ls, 60)
    m, delta, nvec, lo = 7, 3, 4, 0.2
    phi = torch.zeros(nvec * 2 * ctx.half_numel(), dtype=torch.float64 if prec == F64 else torch.float32,
                      device="cuda")
    ops.cheby_recursive_basis(ctx, phi, full_dev(eta, L, prec), lo, lmax, m, delta, nvec, mf)
    got = fulls_canon(phi, L, Ls, nvec)
    want = cheby.recursive_basis(lambda v: dwf.mdagm(U, v, M5, mf), eta, m, delta, nvec, lo, lmax)
    for g, w in zip(got, want):
        err = rel(g, w)
        print(f"recursive_basis prec={prec}: rel err {err:.3e}")
        assert err < tol


def test_chiral_projection(small):
    L, Ls, mf, U, ctx, lmax = small
    v = synth.gaussian_spinor(L, Ls, 61)
    for sign in (1, -1):
        d = full_dev(v, L, F64)
        ops.dwf_chiral_project(ctx, d, d, sign)
        assert rel(dev_to_full_canon(d, L, Ls), coarse.chiral_project(v, sign)) < 1e-15


def oracle_basis(U, L, Ls, block, nvec, seed, mf):
    appA = lambda w: dwf.mdagm(U, w, M5, mf)
    raw = [cheby.cheby_filter(appA, synth.gaussian_spinor(L, Ls, seed + i), 4, 0.5, 70.0)
           for i in range(nvec)]
    half = nvec // 2
    pre = [coarse.chiral_project(v, +1) for v in raw[:half]] + \
          [coarse.chiral_project(v, -1) for v in raw[half:]]
    return pre, coarse.block_orthonormalise(pre, block, [list(range(half)), list(range(half, nvec))])


@pytest.mark.parametrize("L,block,nb", [((4, 4, 4, 4), (2, 2, 2, 2), 4), ((4, 4, 2, 8), (2, 2, 2, 4), 6),
                                        ((8, 4, 4, 4), (4, 4, 2, 2), 8)])
def test_block_orthonormalise_matches_mgs(L, block, nb):
    Ls, mf = 4, 0.1
    U = synth.random_gauge(L, 0.5, 42)
    ctx = ops.Context(L, Ls, M5, U)
    pre, want = oracle_basis(U, L, Ls, block, nb, 100, mf)
    d = fulls_dev(pre, L, F64)
    ops.block_orthonormalise(ctx, d, nb, nb // 2, block)
    got = fulls_canon(d, L, Ls, nb)
    for g, w in zip(got, want):
        assert rel(g, w) < 1e-10
    ctx.close()


@pytest.fixture(scope="module", params=[((4, 4, 4, 4), (2, 2, 2, 2), 4), ((4, 4, 2, 8), (2, 2, 2, 2), 4),
                                        ((8, 4, 4, 4), (4, 2, 2, 2), 6)],
                ids=["4444_b2222", "4428_b2222", "8444_b4222"])
def coarse_case(request):
    L, block, nb = request.param
    Ls, mf = 4, 0.1
    U = synth.random_gauge(L, 0.5, 43)
    ctx = ops.Context(L, Ls, M5, U)
    _, basis = oracle_basis(U, L, Ls, block, nb, 200, mf)
    A = coarse.coarse_build(U, basis, block, M5, mf)  # (9, Tc, Zc, Yc, Xc, nb, nb)
    Aflat = np.moveaxis(A.reshape(9, -1, nb, nb), 0, 1)  # (nc, 9, nb, nb)
    yield L, Ls, block, nb, mf, U, ctx, basis, A, Aflat
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(F64, 1e-12), (F32, 1e-6)])
def test_coarse_build(coarse_case, prec, tol):
    L, Ls, block, nb, mf, U, ctx, basis, A, Aflat = coarse_case
    C = ops.coarse_build(ctx, fulls_dev(basis, L, prec), nb, nb // 2, block, mf)
    got = C.export()
    err = rel(got, Aflat)
    print(f"coarse_build prec={prec}: rel err {err:.3e}")
    assert err < tol
    C.close()


def coarse_vec(A, nb, nrhs, seed):
    nc = A.shape[0]
    return synth.complex_gaussian(seed, (nc, nb, nrhs))


def oracle_coarse_apply(A, v, Lc):
    """v (nc, nb, nrhs) -> stencil apply with the oracle per rhs."""
    nb = v.shape[1]
    Ast = np.moveaxis(A, 1, 0).reshape((9, Lc[3], Lc[2], Lc[1], Lc[0], nb, nb))
    out = np.zeros_like(v)
    for r in range(v.shape[2]):
        vc = v[:, :, r].reshape(Lc[3], Lc[2], Lc[1], Lc[0], nb)
        out[:, :, r] = coarse.coarse_apply(Ast, vc).reshape(-1, nb)
    return out


@pytest.mark.parametrize("nrhs", [1, 3, 8, 32])
def test_coarse_apply(coarse_case, nrhs):
    L, Ls, block, nb, mf, U, ctx, basis, A, Aflat = coarse_case
    C = ops.coarse_build(ctx, fulls_dev(basis, L, F64), nb, nb // 2, block, mf)
    v = coarse_vec(Aflat, nb, nrhs, 7)
    vd = torch.from_numpy(layout.complex_to_real(v, F32).reshape(-1)).cuda()
    out = torch.zeros_like(vd)
    ops.coarse_apply(C, out, vd, nrhs)
    got = layout.real_to_complex(out.double().cpu().numpy()).reshape(v.shape)
    want = oracle_coarse_apply(C.export(), v, C.Lc)
    assert rel(got, want) < 1e-6
    C.close()


def test_coarse_solve(coarse_case):
    L, Ls, block, nb, mf, U, ctx, basis, A, Aflat = coarse_case
    C = ops.coarse_build(ctx, fulls_dev(basis, L, F64), nb, nb // 2, block, mf)
    r = coarse_vec(Aflat, nb, 1, 8)[:, :, 0]
    rd = torch.from_numpy(layout.complex_to_real(r, F32).reshape(-1)).cuda()
    e = torch.zeros_like(rd)
    it = ops.coarse_solve(C, e, rd, 1e-5, 2000)
    assert it > 0
    eg = layout.real_to_complex(e.double().cpu().numpy()).reshape(r.shape)
    dense = coarse.coarse_dense_from_stencil(np.moveaxis(C.export(), 1, 0).reshape(
        (9,) + tuple(C.Lc[::-1]) + (nb, nb)))
    # the stopping rule bounds the normal residual |A^2 e - A r| <= 1e-5 |A r|
    Ar = dense @ r.ravel()
    assert np.linalg.norm(dense @ (dense @ eg.ravel()) - Ar) <= 2e-5 * np.linalg.norm(Ar)
    # and the oracle's CG on A^2 with the same rule reaches the same solution
    e_or, it_or = coarse.coarse_cgnr(np.moveaxis(C.export(), 1, 0).reshape((9,) + tuple(C.Lc[::-1]) + (nb, nb)),
                                     r.reshape(tuple(C.Lc[::-1]) + (nb,)), 1e-5, 2000)
    assert abs(it - it_or) <= 4
    want = np.linalg.solve(dense, r.ravel())
    assert rel(eg.ravel(), want) < 10 * rel(e_or.ravel(), want) + 1e-5
    C.close()


def test_restrict_prolong(coarse_case):
    L, Ls, block, nb, mf, U, ctx, basis, A, Aflat = coarse_case
    bd = fulls_dev(basis, L, F32)
    psi = synth.gaussian_spinor(L, Ls, 9)
    out = torch.zeros(2 * Aflat.shape[0] * nb, dtype=torch.float32, device="cuda")
    ops.dwf_restrict(ctx, out, full_dev(psi, L, F32), bd, nb, block)
    got = layout.real_to_complex(out.double().cpu().numpy()).reshape(-1, nb)
    want = coarse.restrict(basis, psi, block).reshape(-1, nb)
    assert rel(got, want) < 1e-6
    ec = synth.complex_gaussian(10, want.shape)
    ed = torch.from_numpy(layout.complex_to_real(ec, F32).reshape(-1)).cuda()
    fine = ctx.new_full(F32)
    ops.dwf_prolong(ctx, fine, ed, bd, nb, block)
    Lc = [L[m] // block[m] for m in range(4)]
    wantf = coarse.prolong(basis, ec.reshape(Lc[3], Lc[2], Lc[1], Lc[0], nb), block)
    assert rel(dev_to_full_canon(fine, L, Ls), wantf) < 1e-6


# ---------------------------------------------------------------- full setup, smoother, V-cycle, solve
@pytest.fixture(scope="module")
def mg_case():
    L, Ls, mf = (4, 4, 4, 4), 4, 0.05
    block, nb = (2, 2, 2, 2), 8
    U = synth.random_gauge(L, 0.5, 51)
    ctx = ops.Context(L, Ls, M5, U)
    etas = [synth.gaussian_spinor(L, Ls, 600 + i) for i in range(nb)]
    p = ops.mg_params(block, nb, mf, subspace_mode=SUBSPACE_BATCH, lambda_lo=0.5, lambda_max=70.0,
                      filter_order=4, smooth=(0.5, 60.0, 6), coarse_tol=0.02, coarse_maxiter=500,
                      nkrylov=8, maxiter=200)
    G = ops.MG(ctx, p, fulls_dev(etas, L, F64))
    yield L, Ls, mf, block, nb, U, ctx, etas, p, G
    G.close()
    ctx.close()


def test_mg_setup_basis_matches_oracle(mg_case):
    L, Ls, mf, block, nb, U, ctx, etas, p, G = mg_case
    appA = lambda w: dwf.mdagm(U, w, M5, mf)
    raw = [cheby.cheby_filter(appA, e, 4, 0.5, 70.0) for e in etas]
    raw = [v / np.sqrt(dwf.norm2(v)) for v in raw]
    pre = [coarse.chiral_project(v, +1) for v in raw[:nb // 2]] + \
          [coarse.chiral_project(v, -1) for v in raw[nb // 2:]]
    want = coarse.block_orthonormalise(pre, block, [list(range(nb // 2)), list(range(nb // 2, nb))])
    got = fulls_canon(G.basis(), L, Ls, nb)
    for g, w in zip(got, want):
        assert rel(g, w) < 1e-5


def test_mg_smoother(mg_case):
    L, Ls, mf, block, nb, U, ctx, etas, p, G = mg_case
    r = synth.gaussian_spinor(L, Ls, 70)
    out = ctx.new_full(F32)
    ops.mg_smooth(G, out, full_dev(r, L, F32))
    appH = lambda w: dwf.hdw(U, w, M5, mf)
    want, nA = cheby.smoother_apply(appH, appH, r, 0.5, 60.0, 6)
    assert rel(dev_to_full_canon(out, L, Ls), want) < 2e-5


def test_mg_vcycle(mg_case):
    """V(1,1) against the oracle's sequence on the GPU's own (exported) basis.
    Both coarse solves run the same CG on A^2 to a relative normal residual of
    1e-6 (FP32 on the GPU, FP64 in the oracle), so the two corrections differ
    by about 1e-6 times the coarse condition number."""
    L, Ls, mf, block, nb, U, ctx, etas, p, G = mg_case
    p2 = ops.mg_params(block, nb, mf, subspace_mode=SUBSPACE_BATCH, lambda_lo=0.5, lambda_max=70.0,
                       filter_order=4, smooth=(0.5, 60.0, 6), coarse_tol=1e-6, coarse_maxiter=2000)
    G2 = ops.MG(ctx, p2, fulls_dev(etas, L, F64))
    basis = fulls_canon(G2.basis(), L, Ls, nb)
    A = coarse.coarse_build(U, basis, block, M5, mf)
    r = synth.gaussian_spinor(L, Ls, 71)
    out = ctx.new_full(F32)
    ops.mg_precondition(G2, out, full_dev(r, L, F32))
    appH = lambda w: dwf.hdw(U, w, M5, mf)
    want = mg.vcycle(appH, r, basis, A, block, (0.5, 60.0, 6), 1e-6, 5000, mg.MGCounter())
    got = dev_to_full_canon(out, L, Ls)
    assert rel(got, want) < 1e-3
    # the preconditioned residual is smaller than the residual itself
    assert np.sqrt(dwf.norm2(r - appH(got))) < np.sqrt(dwf.norm2(r))
    G2.close()


@pytest.mark.parametrize("host", [False, True])
def test_mg_solve(mg_case, host):
    L, Ls, mf, block, nb, U, ctx, etas, p, G = mg_case
    b = synth.gaussian_spinor(L, Ls, 72)
    tol = 1e-8
    if host:
        bh = layout.complex_to_real(layout.to_full(b, L), F64)
        xh = np.zeros_like(bh)
        st = ops.mg_solve(G, xh, bh, tol)
        x = layout.from_full(layout.real_to_complex(xh).reshape(2, -1, 4, 3, Ls), L)
    else:
        bd = full_dev(b, L, F64)
        xd = torch.zeros_like(bd)
        st = ops.mg_solve(G, xd, bd, tol)
        x = dev_to_full_canon(xd, L, Ls)
    res = krylov.true_residual(U, x, b, M5, mf)
    assert res <= tol * 1.01, st
    assert st["true_residual"] == pytest.approx(res, rel=1e-3, abs=1e-14)
    xr, _, _ = krylov.rbcg_solve(U, b, M5, mf, 1e-13)
    assert rel(x, xr) < 1e-6
    assert st["coarse_iterations"] > 0 and st["fine_matmuls"] > 0


def test_mg_solve_graph_replay_is_identical(mg_case):
    """The V-cycle replayed from a CUDA graph runs the same kernels on the
    same data as plain launches: same outer and coarse iteration counts and
    a bit-identical solution; the graph solve reports its replays."""
    L, Ls, mf, block, nb, U, ctx, etas, p, G = mg_case
    b = full_dev(synth.gaussian_spinor(L, Ls, 73), L, F64)
    runs = []
    for graph in (True, False):
        pg = ops.mg_params(block, nb, mf, subspace_mode=SUBSPACE_BATCH, lambda_lo=0.5, lambda_max=70.0,
                           filter_order=4, smooth=(0.5, 60.0, 6), coarse_tol=0.02, coarse_maxiter=500,
                           nkrylov=8, maxiter=200, graph=graph)
        Gg = ops.MG(ctx, pg, fulls_dev(etas, L, F64))
        x = torch.zeros_like(b)
        st = ops.mg_solve(Gg, x, b, 1e-8)
        runs.append((st, x.clone()))
        Gg.close()
    (sg, xg), (sp, xp) = runs
    assert sg["graph_replays"] == sg["iterations"] - 1 and sg["graph_replays"] > 0
    assert sp["graph_replays"] == 0
    assert (sg["iterations"], sg["coarse_iterations"]) == (sp["iterations"], sp["coarse_iterations"])
    assert sg["fine_matmuls"] == sp["fine_matmuls"]
    assert torch.equal(xg, xp)


@pytest.mark.parametrize("nrhs,L", [(16, (4, 4, 4, 8)), (32, (4, 4, 4, 8)), (64, (4, 4, 4, 8)),
                                     (32, (8, 8, 16, 16))])
def test_coarse_apply_tensor_cores(nrhs, L):
    """tcgen05 TF32 coarse stencil (nb = 32) against the oracle apply of the
    exported FP64 operator.  TF32 rounds each input to 11 significant bits
    (relative error <= 2^-11 = 4.9e-4); with FP32 accumulation of 576 terms of
    random sign the norm-wise error is ~1e-3, so the bound is 3e-3.  The
    8x8x16x16 lattice has 1024 coarse sites = 512 site pairs, more than one
    pair per CTA of the persistent kernel (both accumulators reused)."""
    from paper_2103_05034_gb300._lib import TF32
    Ls, mf, block, nb = 4, 0.1, (2, 2, 2, 2), 32
    U = synth.random_gauge(L, 0.5, 44)
    ctx = ops.Context(L, Ls, M5, U)
    vecs = [coarse.chiral_project(synth.gaussian_spinor(L, Ls, 300 + i), 1 if i < nb // 2 else -1)
            for i in range(nb)]
    d = fulls_dev(vecs, L, F64)
    ops.block_orthonormalise(ctx, d, nb, nb // 2, block)
    C = ops.coarse_build(ctx, d, nb, nb // 2, block, mf)
    v = synth.complex_gaussian(9, (C.nc, nb, nrhs))
    vd = torch.from_numpy(layout.complex_to_real(v, F32).reshape(-1)).cuda()
    out = torch.zeros_like(vd)
    ops.coarse_apply(C, out, vd, nrhs, prec=TF32)
    got = layout.real_to_complex(out.double().cpu().numpy()).reshape(v.shape)
    want = oracle_coarse_apply(C.export(), v, C.Lc)
    assert rel(got, want) < 3e-3
    # and the FP32 CUDA-core path on the same operator
    out32 = torch.zeros_like(vd)
    ops.coarse_apply(C, out32, vd, nrhs)
    got32 = layout.real_to_complex(out32.double().cpu().numpy()).reshape(v.shape)
    assert rel(got32, want) < 1e-6
    # a second call reuses the arranged operator
    out.zero_()
    ops.coarse_apply(C, out, vd, nrhs, prec=TF32)
    assert rel(layout.real_to_complex(out.double().cpu().numpy()).reshape(v.shape), want) < 3e-3
    # the applies are asynchronous; no bounded wait gave up in any of them
    ops.coarse_apply_status(C)
    C.close()
    ctx.close()


def test_coarse_apply_tensor_cores_rejects_unsupported_shapes(coarse_case):
    from paper_2103_05034_gb300._lib import DWFError, TF32
    L, Ls, block, nb, mf, U, ctx, basis, A, Aflat = coarse_case
    C = ops.coarse_build(ctx, fulls_dev(basis, L, F64), nb, nb // 2, block, mf)
    v = torch.zeros(2 * C.nc * nb * 32, dtype=torch.float32, device="cuda")
    with pytest.raises(DWFError):  # nb != 32 here
        ops.coarse_apply(C, v.clone(), v, 32, prec=TF32)
    C.close()


# ---------------------------------------------------------------- the benchmarked shapes
def _ortho_basis_oracle(L, Ls, block, nb, seed):
    """Chirality-projected Gaussians orthonormalised per (block, chirality) by
    the oracle (MGS2): the same FP64 basis goes to both sides."""
    vecs = [coarse.chiral_project(synth.gaussian_spinor(L, Ls, seed + i), 1 if i < nb // 2 else -1)
            for i in range(nb)]
    return coarse.block_orthonormalise(vecs, block, [list(range(nb // 2)), list(range(nb // 2, nb))])


@pytest.mark.parametrize("Ls,nb", [(16, 32), (24, 8), (8, 8)])
@pytest.mark.parametrize("prec,tol", [(F64, 1e-12), (F32, 1e-6)])
def test_coarse_build_at_benchmark_ls(Ls, nb, prec, tol):
    """The face-split hopping kernels k_face_hop<P, Ls> at Ls = 8, 16, 24 and
    the 32-vector build (the benchmark's multigrid shape) against the oracle's
    9-point stencil; the F32 bound is c12's FP32 operator bound (FP32 basis and
    hops, FP64 block sums)."""
    L, block, mf = (4, 4, 4, 4), (2, 2, 2, 2), 0.1
    U = synth.random_gauge(L, 0.5, 45)
    ctx = ops.Context(L, Ls, M5, U)
    basis = _ortho_basis_oracle(L, Ls, block, nb, 400)
    A = coarse.coarse_build(U, basis, block, M5, mf)
    Aflat = np.moveaxis(A.reshape(9, -1, nb, nb), 0, 1)
    C = ops.coarse_build(ctx, fulls_dev(basis, L, prec), nb, nb // 2, block, mf)
    err = rel(C.export(), Aflat)
    print(f"coarse_build Ls={Ls} nb={nb} prec={prec}: rel err {err:.3e}")
    assert err < tol
    C.close()
    ctx.close()


@pytest.mark.parametrize("nb", [32, 64])
def test_coarse_solve_fixed_width_kernels(nb):
    """The persistent coarse CG with the basis width fixed at compile time
    (k_coarse_cg<32>, which the benchmark's multigrid runs, and <64>): 8^4 x
    Ls 4 with 2^4 blocks gives 256 coarse sites, each CTA owning many rows.
    Same checks as test_coarse_solve: the normal residual bound, the oracle's
    iteration count for the same rule on the same (exported) operator, and
    the exact solution."""
    L, Ls, block, mf = (8, 8, 8, 8), 4, (2, 2, 2, 2), 0.1
    U = synth.random_gauge(L, 0.5, 46)
    ctx = ops.Context(L, Ls, M5, U)
    # the basis (an input of the coarse solve) is built on the GPU: Gaussians
    # filtered towards the low modes of D^dag D, chirality-projected and
    # block-orthonormalised, so that the coarse operator is ill-conditioned
    # enough for the CG to take many iterations
    g = fulls_dev([synth.gaussian_spinor(L, Ls, 500 + i) for i in range(nb)], L, F64)
    d = torch.zeros_like(g)
    ops.cheby_filter(ctx, d, g, nb, 0.5, 70.0, 8, mf)
    half = d.numel() // 2
    ops.dwf_chiral_project(ctx, d[:half], d[:half], 1, nb // 2)
    ops.dwf_chiral_project(ctx, d[half:], d[half:], -1, nb // 2)
    ops.block_orthonormalise(ctx, d, nb, nb // 2, block)
    C = ops.coarse_build(ctx, d, nb, nb // 2, block, mf)
    Ast = np.moveaxis(C.export(), 1, 0).reshape((9,) + tuple(C.Lc[::-1]) + (nb, nb))
    r = synth.complex_gaussian(8, (C.nc, nb))
    rd = torch.from_numpy(layout.complex_to_real(r, F32).reshape(-1)).cuda()
    e = torch.zeros_like(rd)
    tol = 1e-5
    it = ops.coarse_solve(C, e, rd, tol, 5000)
    eg = layout.real_to_complex(e.double().cpu().numpy()).reshape(r.shape)
    Ar = coarse.coarse_apply(Ast, r.reshape(tuple(C.Lc[::-1]) + (nb,)))
    AAe = coarse.coarse_apply(Ast, coarse.coarse_apply(Ast, eg.reshape(Ar.shape)))
    assert np.linalg.norm(AAe - Ar) <= 2 * tol * np.linalg.norm(Ar)
    e_or, it_or = coarse.coarse_cgnr(Ast, r.reshape(Ar.shape), tol, 5000)
    print(f"coarse_solve nb={nb}: {it} iterations (oracle {it_or})")
    assert abs(it - it_or) <= max(4, it_or // 20)
    # the exact solution, from the oracle's CG run far past the tolerance (a
    # dense solve of 256 x nb unknowns is too large here)
    want, _ = coarse.coarse_cgnr(Ast, r.reshape(Ar.shape), 1e-12, 50000)
    assert rel(eg.ravel(), want.ravel()) < 10 * rel(e_or.ravel(), want.ravel()) + 1e-5
    C.close()
    ctx.close()


def test_mg_solve_at_ls16():
    """The whole HDCR solve at Ls = 16 (the benchmark's fifth-dimension
    extent; every other multigrid test runs Ls = 4): FP64 true residual and
    the oracle's red-black solution."""
    L, Ls, mf = (4, 4, 4, 4), 16, 0.05
    block, nb = (2, 2, 2, 2), 8
    U = synth.random_gauge(L, 0.5, 52)
    ctx = ops.Context(L, Ls, M5, U)
    etas = [synth.gaussian_spinor(L, Ls, 700 + i) for i in range(nb)]
    p = ops.mg_params(block, nb, mf, subspace_mode=SUBSPACE_BATCH, lambda_lo=0.5, lambda_max=70.0,
                      filter_order=4, smooth=(0.5, 60.0, 6), coarse_tol=0.02, coarse_maxiter=500,
                      nkrylov=8, maxiter=300)
    G = ops.MG(ctx, p, fulls_dev(etas, L, F64))
    b = synth.gaussian_spinor(L, Ls, 74)
    bd = full_dev(b, L, F64)
    xd = torch.zeros_like(bd)
    st = ops.mg_solve(G, xd, bd, 1e-8)
    x = dev_to_full_canon(xd, L, Ls)
    res = krylov.true_residual(U, x, b, M5, mf)
    assert res <= 1e-8 * 1.01, st
    xr, _, _ = krylov.rbcg_solve(U, b, M5, mf, 1e-13)
    assert rel(x, xr) < 1e-6
    G.close()
    ctx.close()


# ---------------------------------------------------------------- red-black coarse solve
def test_coarse_solve_rb(coarse_case):
    """coarse_solve_rb (CG on the even Schur complement squared) against the
    oracle's coarse_rb_solve on the exported operator: the same iteration
    count for the same stopping rule, and the dense solution of A e = r.  The
    4428 blocking has a coarse extent of 1 (odd): the call must refuse it."""
    from paper_2103_05034_gb300._lib import DWFError
    L, Ls, block, nb, mf, U, ctx, basis, A, Aflat = coarse_case
    C = ops.coarse_build(ctx, fulls_dev(basis, L, F64), nb, nb // 2, block, mf)
    r = coarse_vec(Aflat, nb, 1, 8)[:, :, 0]
    rd = torch.from_numpy(layout.complex_to_real(r, F32).reshape(-1)).cuda()
    e = torch.zeros_like(rd)
    if any(n % 2 for n in C.Lc):
        with pytest.raises(DWFError):
            ops.coarse_solve_rb(C, e, rd, 1e-5, 2000)
        C.close()
        return
    it = ops.coarse_solve_rb(C, e, rd, 1e-5, 2000)
    Ast = np.moveaxis(C.export(), 1, 0).reshape((9,) + tuple(C.Lc[::-1]) + (nb, nb))
    e_or, it_or = coarse.coarse_rb_solve(Ast, r.reshape(tuple(C.Lc[::-1]) + (nb,)), 1e-5, 2000)
    assert abs(it - it_or) <= max(4, it_or // 20), (it, it_or)
    eg = layout.real_to_complex(e.double().cpu().numpy()).reshape(r.shape)
    dense = coarse.coarse_dense_from_stencil(Ast)
    want = np.linalg.solve(dense, r.ravel())
    assert rel(eg.ravel(), want) < 10 * rel(e_or.ravel(), want) + 1e-5
    C.close()


@pytest.mark.parametrize("nb", [32, 64])
def test_coarse_solve_rb_fixed_width(nb):
    """The red-black coarse CG with nb fixed at compile time (32, 64) on a 4^4
    coarse lattice (8^4 x Ls 4, 2^4 blocks), filtered basis: iterations against
    the oracle's red-black CG, the solution against the oracle's plain CG on
    A^2 run far past the tolerance, and fewer iterations than the plain CG on
    A^2 for the same relative tolerance."""
    L, Ls, block, mf = (8, 8, 8, 8), 4, (2, 2, 2, 2), 0.01
    U = synth.random_gauge(L, 0.5, 47)
    ctx = ops.Context(L, Ls, M5, U)
    g = fulls_dev([synth.gaussian_spinor(L, Ls, 520 + i) for i in range(nb)], L, F64)
    d = torch.zeros_like(g)
    ops.cheby_filter(ctx, d, g, nb, 0.2, 70.0, 12, mf)
    half = d.numel() // 2
    ops.dwf_chiral_project(ctx, d[:half], d[:half], 1, nb // 2)
    ops.dwf_chiral_project(ctx, d[half:], d[half:], -1, nb // 2)
    ops.block_orthonormalise(ctx, d, nb, nb // 2, block)
    C = ops.coarse_build(ctx, d, nb, nb // 2, block, mf)
    Ast = np.moveaxis(C.export(), 1, 0).reshape((9,) + tuple(C.Lc[::-1]) + (nb, nb))
    r = synth.complex_gaussian(11, (C.nc, nb))
    rd = torch.from_numpy(layout.complex_to_real(r, F32).reshape(-1)).cuda()
    e = torch.zeros_like(rd)
    tol = 1e-5
    it = ops.coarse_solve_rb(C, e, rd, tol, 5000)
    e_or, it_or = coarse.coarse_rb_solve(Ast, r.reshape(tuple(C.Lc[::-1]) + (nb,)), tol, 5000)
    print(f"coarse_solve_rb nb={nb}: {it} iterations (oracle {it_or})")
    assert abs(it - it_or) <= max(4, it_or // 20)
    eg = layout.real_to_complex(e.double().cpu().numpy()).reshape(r.shape)
    want, _ = coarse.coarse_cgnr(Ast, r.reshape(tuple(C.Lc[::-1]) + (nb,)), 1e-12, 50000)
    assert rel(eg.ravel(), want.ravel()) < 10 * rel(e_or.ravel(), want.ravel()) + 1e-5
    e2 = torch.zeros_like(rd)
    it_plain = ops.coarse_solve(C, e2, rd, tol, 5000)
    print(f"  plain CG on A^2: {it_plain} iterations")
    assert it < it_plain
    C.close()
    ctx.close()


def test_mg_solve_with_red_black_coarse_solver(mg_case):
    """The HDCR solve with the red-black coarse solver reaches the tolerance
    and the oracle's solution, as the plain coarse CG does."""
    from paper_2103_05034_gb300._lib import COARSE_RB
    L, Ls, mf, block, nb, U, ctx, etas, p, G = mg_case
    prb = ops.mg_params(block, nb, mf, subspace_mode=SUBSPACE_BATCH, lambda_lo=0.5, lambda_max=70.0,
                        filter_order=4, smooth=(0.5, 60.0, 6), coarse_tol=0.02, coarse_maxiter=500,
                        nkrylov=8, maxiter=200, coarse_solver=COARSE_RB)
    Grb = ops.MG(ctx, prb, fulls_dev(etas, L, F64))
    b = synth.gaussian_spinor(L, Ls, 75)
    bd = full_dev(b, L, F64)
    xd = torch.zeros_like(bd)
    st = ops.mg_solve(Grb, xd, bd, 1e-8)
    x = dev_to_full_canon(xd, L, Ls)
    assert krylov.true_residual(U, x, b, M5, mf) <= 1e-8 * 1.01, st
    xr, _, _ = krylov.rbcg_solve(U, b, M5, mf, 1e-13)
    assert rel(x, xr) < 1e-6
    assert st["coarse_iterations"] > 0 and st["graph_replays"] > 0
    Grb.close()


# ---------------------------------------------------------------- coarse deflation
@pytest.fixture(scope="module")
def defl_case():
    """A 4^4-site coarse lattice (8^4 x Ls 16, 2^4 blocks) with a 16-vector
    basis filtered towards the low modes and a light mass (at Ls = 16 the
    residual mass is small): an operator whose A^2 spans several decades."""
    L, Ls, block, mf, nb = (8, 8, 8, 8), 16, (2, 2, 2, 2), 0.001, 16
    U = synth.random_gauge(L, 0.5, 48, ape_steps=2)
    ctx = ops.Context(L, Ls, M5, U)
    g = fulls_dev([synth.gaussian_spinor(L, Ls, 540 + i) for i in range(nb)], L, F64)
    d = torch.zeros_like(g)
    ops.cheby_filter(ctx, d, g, nb, 0.05, 70.0, 24, mf)
    half = d.numel() // 2
    ops.dwf_chiral_project(ctx, d[:half], d[:half], 1, nb // 2)
    ops.dwf_chiral_project(ctx, d[half:], d[half:], -1, nb // 2)
    ops.block_orthonormalise(ctx, d, nb, nb // 2, block)
    C = ops.coarse_build(ctx, d, nb, nb // 2, block, mf)
    Ast = np.moveaxis(C.export(), 1, 0).reshape((9,) + tuple(C.Lc[::-1]) + (nb, nb))
    yield ctx, C, Ast, nb
    C.close()
    ctx.close()


def test_coarse_deflation_ritz_pairs(defl_case):
    """Chebyshev-preconditioned Lanczos on A^2 (Sec. 3.5) from the same start
    vector as the oracle's cheby_lanczos: the lowest Ritz values agree (FP32
    Lanczos vectors against FP64), and every GPU pair is an eigenpair of the
    exported operator's A^2 to a small residual."""
    ctx, C, Ast, nb = defl_case
    nev, nk, order, lo = 8, 60, 8, 0.05
    v0 = synth.complex_gaussian(13, (C.nc, nb))
    v0d = torch.from_numpy(layout.complex_to_real(v0, F32).reshape(-1)).cuda()
    shape = tuple(C.Lc[::-1]) + (nb,)
    appAA = lambda v: coarse.coarse_apply(Ast, coarse.coarse_apply(Ast, v.reshape(shape))).reshape(v.shape)
    lam = 0.0
    v = v0.ravel() / np.linalg.norm(v0)
    for _ in range(30):  # the oracle's lambda_max from the same power method
        w = appAA(v)
        lam = np.linalg.norm(w)
        v = w / lam
    lmax = 1.1 * lam
    th = ops.coarse_deflate(C, v0d, nev, nk, order, lo, lmax)
    th_or, V_or = coarse.cheby_lanczos(appAA, v0.ravel(), nev, nk, order, lo, lmax)
    print("GPU Ritz values", np.array(th)[:4], "oracle", th_or[:4])
    assert np.allclose(np.sort(th)[:4], np.sort(th_or)[:4], rtol=1e-3)
    V, thinv = ops.coarse_export_deflation(C)
    Vm = V.reshape(nev, -1)
    # orthonormal Ritz vectors whose Rayleigh quotients are the Ritz values
    assert np.abs(Vm.conj() @ Vm.T - np.eye(nev)).max() < 1e-4
    for i in range(nev):
        assert np.vdot(Vm[i], appAA(Vm[i])).real == pytest.approx(1.0 / thinv[i], rel=1e-4)
    # and the lowest pair approximates an eigenpair of A^2 (its residual is
    # small on the scale of the spectrum)
    r = appAA(Vm[0]) - Vm[0] / thinv[0]
    print("lowest Ritz pair residual / lambda_max:", np.linalg.norm(r) / lmax)
    assert np.linalg.norm(r) <= 5e-2 * lmax
    ops.coarse_deflate(C, None, 0, 0, 0, 0.0)


@pytest.fixture(scope="module")
def mg16():
    """The multigrid of the 16^3 x 32 x 16 workload (recursive subspace with
    m = 300, Delta = 60; 4^4 x Ls blocks, 16 + 16 vectors): its coarse
    operator has the low modes the deflation is for."""
    from paper_2103_05034_gb300._lib import SUBSPACE_RECURSIVE
    name = "dwf_16x16x16x32_ls16"
    w = synth.WORKLOADS[name]
    L, Ls, mf = w["L"], w["Ls"], w["mf"]
    ctx = ops.Context(L, Ls, M5, synth.workload_gauge(name))
    eta = full_dev(synth.gaussian_spinor(L, Ls, synth.SEED_BASIS), L, F64)
    p = ops.mg_params((4, 4, 4, 4), 32, mf, subspace_mode=SUBSPACE_RECURSIVE, lambda_lo=0.05, lambda_max=80.0,
                      filter_order=300, delta=60, smooth=(0.05, 80.0, 40), coarse_tol=2e-3)
    G = ops.MG(ctx, p, eta)
    yield ctx, G
    G.close()
    ctx.close()


def test_coarse_deflated_solve(mg16):
    """The coarse CG started from the deflation guess against the oracle's
    coarse_deflated_cgnr with the GPU's own (exported) Ritz pairs, on the
    16^3 multigrid's coarse operator: the same iteration count, the solution
    (against the oracle's deflated CG run far past the tolerance), and far
    fewer iterations than without deflation."""
    ctx, G = mg16
    C = G.coarse
    nb = C.nb
    Ast = np.moveaxis(C.export(), 1, 0).reshape((9,) + tuple(C.Lc[::-1]) + (nb, nb))
    v0 = synth.complex_gaussian(14, (C.nc, nb))
    v0d = torch.from_numpy(layout.complex_to_real(v0, F32).reshape(-1)).cuda()
    ops.coarse_deflate(C, v0d, 32, 96, 10, 0.05)
    V, thinv = ops.coarse_export_deflation(C)
    shape = tuple(C.Lc[::-1]) + (nb,)
    Vs = [V[i].reshape(shape) for i in range(len(thinv))]
    r = synth.complex_gaussian(15, (C.nc, nb))
    rd = torch.from_numpy(layout.complex_to_real(r, F32).reshape(-1)).cuda()
    tol = 1e-5
    e = torch.zeros_like(rd)
    it = ops.coarse_solve(C, e, rd, tol, 5000)
    e_or, it_or = coarse.coarse_deflated_cgnr(Ast, r.reshape(shape), 1.0 / thinv, Vs, tol, 5000)
    ops.coarse_deflate(C, None, 0, 0, 0, 0.0)
    e2 = torch.zeros_like(rd)
    it_plain = ops.coarse_solve(C, e2, rd, tol, 5000)
    print(f"deflated coarse CG: {it} iterations (oracle {it_or}), undeflated {it_plain}")
    assert abs(it - it_or) <= max(4, it_or // 10)
    assert 2 * it < it_plain
    eg = layout.real_to_complex(e.double().cpu().numpy()).reshape(r.shape)
    want, _ = coarse.coarse_deflated_cgnr(Ast, r.reshape(shape), 1.0 / thinv, Vs, 1e-11, 20000)
    assert rel(eg.ravel(), want.ravel()) < 10 * rel(e_or.ravel(), want.ravel()) + 1e-5


def test_mg_solve_with_deflated_coarse_solver(mg_case):
    from paper_2103_05034_gb300._lib import COARSE_DEFLATED
    L, Ls, mf, block, nb, U, ctx, etas, p, G = mg_case
    pd = ops.mg_params(block, nb, mf, subspace_mode=SUBSPACE_BATCH, lambda_lo=0.5, lambda_max=70.0,
                       filter_order=4, smooth=(0.5, 60.0, 6), coarse_tol=0.02, coarse_maxiter=500,
                       nkrylov=8, maxiter=200, coarse_solver=COARSE_DEFLATED, deflation=(8, 24, 8, 0.5))
    Gd = ops.MG(ctx, pd, fulls_dev(etas, L, F64))
    b = synth.gaussian_spinor(L, Ls, 76)
    bd = full_dev(b, L, F64)
    xd = torch.zeros_like(bd)
    st = ops.mg_solve(Gd, xd, bd, 1e-8)
    x = dev_to_full_canon(xd, L, Ls)
    assert krylov.true_residual(U, x, b, M5, mf) <= 1e-8 * 1.01, st
    xr, _, _ = krylov.rbcg_solve(U, b, M5, mf, 1e-13)
    assert rel(x, xr) < 1e-6
    Gd.close()


@pytest.mark.parametrize("prec_name", ["f32", "tf32"])
def test_coarse_solve_multi(mg16, prec_name):
    """CG on A^2 for 16 right-hand sides at once on the 16^3 multigrid's
    coarse operator (the tensor-core stencil's solve-path caller): every
    solution satisfies the stopping rule under the exported FP64 operator
    (with the TF32 operator's error of about 5e-4 allowed for), and on the
    CUDA cores the first two right-hand sides take the oracle's CG iteration
    counts (to the 8-iteration granularity of the checks)."""
    from paper_2103_05034_gb300._lib import TF32
    ctx, G = mg16
    C = G.coarse
    nb, nrhs = C.nb, 16
    prec = {"f32": F32, "tf32": TF32}[prec_name]
    tol = 1e-4 if prec_name == "f32" else 2e-3
    shape = tuple(C.Lc[::-1]) + (nb,)
    Ast = np.moveaxis(C.export(), 1, 0).reshape((9,) + shape[:4] + (nb, nb))
    r = synth.complex_gaussian(16, (C.nc, nb, nrhs))
    rd = torch.from_numpy(layout.complex_to_real(r, F32).reshape(-1)).cuda()
    e = torch.zeros_like(rd)
    its = ops.coarse_solve_multi(C, e, rd, nrhs, tol, 5000, prec)
    eg = layout.real_to_complex(e.double().cpu().numpy()).reshape(r.shape)
    slack = 1.01 if prec_name == "f32" else 2.0
    for k in range(nrhs):
        Ar = coarse.coarse_apply(Ast, r[:, :, k].reshape(shape))
        res = coarse.coarse_apply(Ast, coarse.coarse_apply(Ast, eg[:, :, k].reshape(shape))) - Ar
        assert np.linalg.norm(res) <= slack * tol * np.linalg.norm(Ar) + (1e-3 if prec_name == "tf32" else 0) * \
            np.linalg.norm(Ar), (k, its[k])
    print(f"coarse_solve_multi {prec_name}: iterations {its}")
    if prec_name == "f32":
        for k in range(2):
            _, it_or = coarse.coarse_cgnr(Ast, r[:, :, k].reshape(shape), tol, 5000)
            slack_it = max(4, it_or // 20)
            assert it_or - slack_it <= its[k] < it_or + 8 + slack_it
