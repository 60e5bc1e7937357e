"""GPU parity of the fine operators and the red-black CG through the C ABI,
against the FP64 oracle (Sec. 2 and Sec. 5.1 of arXiv:2103.05034).

Tolerances (norm-wise relative): FP64 1e-12, FP32 1e-6 (operators with FP32
arithmetic on O(1) data: ~10 roundings per output of relative size 6e-8),
FP16 storage 2e-3 (one rounding of input and output at 4.9e-4 each, summed
over 8 neighbours)."""
import numpy as np
import pytest
import torch

import synth
from oracle import dwf, krylov
from paper_2103_05034_gb300 import _lib, ops
from paper_2103_05034_gb300._lib import (DWF_EINVAL, F16S, F32, F64, SOLVE_F64, SOLVE_MIXED_F32,
                                         DWFError)

from gpu_helpers import dev_to_full_canon, dev_to_half, full_dev, half_dev, rel

pytestmark = pytest.mark.gpu
M5 = 1.8
TOL = {F64: 1e-12, F32: 1e-6, F16S: 2e-3}

CASES = [((4, 4, 4, 4), 8), ((2, 2, 2, 6), 8), ((4, 2, 2, 4), 4), ((4, 4, 2, 2), 16),
         ((2, 4, 2, 2), 24)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"L{'x'.join(map(str, c[0]))}_Ls{c[1]}")
def case(request):
    L, Ls = request.param
    U = synth.random_gauge(L, 0.5, 7)
    ctx = ops.Context(L, Ls, M5, U)
    yield L, Ls, U, ctx
    ctx.close()


@pytest.mark.parametrize("prec", [F64, F32, F16S])
@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_dhop_parity(case, prec, dagger, out_parity):
    L, Ls, U, ctx = case
    psi = synth.gaussian_spinor(L, Ls, 11)
    src = dwf.project_parity(psi, L, 1 - out_parity)
    inp = half_dev(psi, L, 1 - out_parity, prec)
    out = torch.zeros_like(inp)
    ops.dwf_dhop(ctx, out, inp, out_parity, dagger)
    want = dwf.dhop(U, src, dag=bool(dagger))
    from paper_2103_05034_gb300 import layout
    want = layout.to_half(want, L, out_parity)
    assert rel(dev_to_half(out, Ls), want) < TOL[prec]


def test_dhop_batched(case):
    L, Ls, U, ctx = case
    nrhs = 3
    psis = [synth.gaussian_spinor(L, Ls, 20 + i) for i in range(nrhs)]
    inp = torch.cat([half_dev(p, L, 1, F32) for p in psis])
    out = torch.zeros_like(inp)
    ops.dwf_dhop(ctx, out, inp, 0, 0, nrhs=nrhs)
    from paper_2103_05034_gb300 import layout
    got = dev_to_half(out, Ls).reshape(nrhs, -1, 4, 3, Ls)
    for i, p in enumerate(psis):
        want = layout.to_half(dwf.dhop(U, dwf.project_parity(p, L, 1)), L, 0)
        assert rel(got[i], want) < TOL[F32]


@pytest.mark.parametrize("prec", [F64, F32])
@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("mf", [0.01, 0.3])
def test_mooee_and_inverse(case, prec, dagger, mf):
    L, Ls, U, ctx = case
    from paper_2103_05034_gb300 import layout
    psi = dwf.project_parity(synth.gaussian_spinor(L, Ls, 12), L, 0)
    inp = half_dev(psi, L, 0, prec)
    out = torch.zeros_like(inp)
    ops.dwf_mooee(ctx, out, inp, mf, dagger)
    want = layout.to_half(dwf.mooee(psi, M5, mf, dag=bool(dagger)), L, 0)
    assert rel(dev_to_half(out, Ls), want) < TOL[prec]
    ops.dwf_mooee_inv(ctx, out, inp, mf, dagger)
    want = layout.to_half(dwf.mooee_inv(psi, M5, mf, dag=bool(dagger)), L, 0)
    assert rel(dev_to_half(out, Ls), want) < TOL[prec]


@pytest.mark.parametrize("prec", [F64, F32])
def test_mpc_and_normal_op(case, prec):
    L, Ls, U, ctx = case
    from paper_2103_05034_gb300 import layout
    mf = 0.05
    psi = dwf.project_parity(synth.gaussian_spinor(L, Ls, 13), L, 0)
    inp = half_dev(psi, L, 0, prec)
    out = torch.zeros_like(inp)
    for dagger, fn in ((0, dwf.mpc), (1, dwf.mpc_dag)):
        ops.dwf_mpc(ctx, out, inp, mf, dagger)
        assert rel(dev_to_half(out, Ls), layout.to_half(fn(U, psi, M5, mf), L, 0)) < TOL[prec]
    ops.dwf_mpcdag_mpc(ctx, out, inp, mf)
    want = layout.to_half(dwf.mpcdag_mpc(U, psi, M5, mf), L, 0)
    assert rel(dev_to_half(out, Ls), want) < TOL[prec]


@pytest.mark.parametrize("prec", [F64, F32])
def test_full_ddw_and_hdw(case, prec):
    L, Ls, U, ctx = case
    mf = 0.02
    psi = synth.gaussian_spinor(L, Ls, 14)
    inp = full_dev(psi, L, prec)
    out = torch.zeros_like(inp)
    for dagger in (0, 1):
        ops.dwf_ddw(ctx, out, inp, mf, dagger)
        want = dwf.ddw(U, psi, M5, mf, dag=bool(dagger))
        assert rel(dev_to_full_canon(out, L, Ls), want) < TOL[prec]
    ops.dwf_hdw(ctx, out, inp, mf)
    assert rel(dev_to_full_canon(out, L, Ls), dwf.hdw(U, psi, M5, mf)) < TOL[prec]


def test_reductions(case):
    L, Ls, U, ctx = case
    a = synth.gaussian_spinor(L, Ls, 15)
    b = synth.gaussian_spinor(L, Ls, 16)
    ad, bd = full_dev(a, L, F64), full_dev(b, L, F64)
    assert abs(ops.dwf_norm2(ctx, ad) - dwf.norm2(a)) < 1e-12 * dwf.norm2(a)
    ip = ops.dwf_cdot(ctx, ad, bd)
    want = dwf.inner(a, b)
    assert abs(ip - want) < 1e-12 * np.sqrt(dwf.norm2(a) * dwf.norm2(b))


@pytest.mark.parametrize("policy", [SOLVE_F64, SOLVE_MIXED_F32, _lib.SOLVE_MIXED_F16])
def test_rbcg_solution_parity(policy):
    """4^4 x Ls=8, U = exp(0.3 i H), M5 = 1.8, mf = 0.01 (the small FP64
    workload): GPU solution vs oracle solution, for FP64, FP32-inner and
    FP16-storage-inner CG (the last two with FP64 reliable updates)."""
    L, Ls, mf = (4, 4, 4, 4), 8, 0.01
    U = synth.random_gauge(L, 0.3, synth.SEED_GAUGE)
    b = synth.gaussian_spinor(L, Ls, synth.SEED_SOURCE)
    ctx = ops.Context(L, Ls, M5, U)
    tol = 1e-10
    bd = full_dev(b, L, F64)
    x = torch.zeros_like(bd)
    st = ops.rbcg_solve(ctx, x, bd, mf, tol, 20000, policy)
    xg = dev_to_full_canon(x, L, Ls)
    res = krylov.true_residual(U, xg, b, M5, mf)
    assert res <= tol * 1.01, st
    assert st["true_residual"] == pytest.approx(res, rel=1e-3, abs=1e-14)
    xr, it, _ = krylov.rbcg_solve(U, b, M5, mf, 1e-13)
    assert rel(xg, xr) < 1e-7
    # blocks of CG iterations replayed from a CUDA graph
    assert st["graph_replays"] > 0
    # iteration counts of the two CGs agree closely in FP64
    if policy == SOLVE_F64:
        xo, it10, _ = krylov.rbcg_solve(U, b, M5, mf, 1e-10)
        assert abs(st["iterations"] - it10) <= 0.05 * it10 + 8
    ctx.close()


@pytest.mark.parametrize("policy", [SOLVE_F64, SOLVE_MIXED_F32])
def test_rbcg2_second_schur_form_matches_oracle(policy):
    """The second Schur form of Table 5 (M2 = M_ee^-1 M_pc, CGNR on M2^dag M2)
    on the small FP64 workload: the GPU solution against the oracle's
    rbcg2_solve, the true residual by the oracle, the FP64 iteration count
    against the oracle's CG on the same operator, and (Table 5) more
    iterations than the first form for the same residual."""
    L, Ls, mf = (4, 4, 4, 4), 8, 0.01
    U = synth.random_gauge(L, 0.3, synth.SEED_GAUGE)
    b = synth.gaussian_spinor(L, Ls, synth.SEED_SOURCE)
    ctx = ops.Context(L, Ls, M5, U)
    tol = 1e-10
    bd = full_dev(b, L, F64)
    x = torch.zeros_like(bd)
    st = ops.rbcg2_solve(ctx, x, bd, mf, tol, 20000, policy)
    xg = dev_to_full_canon(x, L, Ls)
    res = krylov.true_residual(U, xg, b, M5, mf)
    assert res <= tol * 1.01, st
    assert st["true_residual"] == pytest.approx(res, rel=1e-3, abs=1e-14)
    xr, _, _ = krylov.rbcg2_solve(U, b, M5, mf, 1e-13)
    assert rel(xg, xr) < 1e-7
    x1 = torch.zeros_like(bd)
    st1 = ops.rbcg_solve(ctx, x1, bd, mf, tol, 20000, policy)
    assert st["iterations"] >= st1["iterations"]
    if policy == SOLVE_F64:
        # the oracle's CG stops on its recursive normal residual; run it to the
        # GPU's final true residual and compare counts
        _, it2, hist = krylov.rbcg2_solve(U, b, M5, mf, 1e-10)
        assert abs(st["iterations"] - it2) <= 0.1 * it2 + 8
    ctx.close()


@pytest.mark.parametrize("Ls,mf", [(4, 0.05), (8, 0.01)])
def test_rbcg_mixed_reaches_tight_tolerance(Ls, mf):
    """A gauge field (4^4, eps 0.3, seed 43) on which the FP32-inner CG,
    keeping its direction across reliable updates without restoring
    <r, p> = |r|^2, diverged below a true residual of about 1e-6: every
    policy must reach 1e-10."""
    L = (4, 4, 4, 4)
    U = synth.random_gauge(L, 0.3, 43)
    b = synth.gaussian_spinor(L, Ls, 44)
    ctx = ops.Context(L, Ls, M5, U)
    bd = full_dev(b, L, F64)
    for policy in (SOLVE_F64, SOLVE_MIXED_F32, _lib.SOLVE_MIXED_F16):
        x = torch.zeros_like(bd)
        st = ops.rbcg_solve(ctx, x, bd, mf, 1e-10, 5000, policy)
        res = krylov.true_residual(U, dev_to_full_canon(x, L, Ls), b, M5, mf)
        assert res <= 1e-10 * 1.01, (policy, st)
    ctx.close()


def test_cgnr_unpreconditioned_matches_oracle():
    """Full-lattice CGNR without red-black preconditioning (the baseline row
    of the Krylov comparison, Sec. 5.1), FP64: the solution against the
    oracle's, the true residual by the oracle, and the iteration count
    against the oracle's CG on D^dag D (more iterations than red-black CG)."""
    L, Ls, mf, tol = (4, 4, 4, 4), 8, 0.01, 1e-10
    U = synth.random_gauge(L, 0.3, synth.SEED_GAUGE)
    b = synth.gaussian_spinor(L, Ls, synth.SEED_SOURCE)
    ctx = ops.Context(L, Ls, M5, U)
    bd = full_dev(b, L, F64)
    x = torch.zeros_like(bd)
    st = ops.cgnr_solve(ctx, x, bd, mf, tol, 20000)
    xg = dev_to_full_canon(x, L, Ls)
    assert krylov.true_residual(U, xg, b, M5, mf) <= tol * 1.01, st
    xr, it_rb, _ = krylov.rbcg_solve(U, b, M5, mf, 1e-13)
    assert rel(xg, xr) < 1e-7
    rhs = dwf.ddw(U, b, M5, mf, dag=True)
    _, it_lo, _ = krylov.cg(lambda v: dwf.mdagm(U, v, M5, mf), rhs, tol, 20000)
    _, it_hi, _ = krylov.cg(lambda v: dwf.mdagm(U, v, M5, mf), rhs, tol * 1e-3, 20000)
    assert it_lo - 8 <= st["iterations"] <= it_hi + 8, (st, it_lo, it_hi)
    _, it_rb10, _ = krylov.rbcg_solve(U, b, M5, mf, tol)
    assert st["iterations"] > it_rb10
    assert st["fine_matmuls"] >= 2 * st["iterations"]
    # zero source; aliasing rejected
    z = torch.zeros_like(bd)
    assert ops.cgnr_solve(ctx, x, z, mf, tol, 10)["iterations"] == 0 and float(x.abs().max()) == 0.0
    with pytest.raises(DWFError) as e:
        ops.cgnr_solve(ctx, bd, bd, mf, tol, 10)
    assert e.value.code == DWF_EINVAL
    ctx.close()


def test_rbcg_host_buffers():
    L, Ls, mf = (4, 4, 4, 4), 8, 0.05
    U = synth.random_gauge(L, 0.3, 3)
    b = synth.gaussian_spinor(L, Ls, 4)
    ctx = ops.Context(L, Ls, M5, U)
    from paper_2103_05034_gb300 import layout
    bh = layout.complex_to_real(layout.to_full(b, L), F64)
    xh = np.zeros_like(bh)
    st = ops.rbcg_solve(ctx, xh, bh, mf, 1e-9, 5000, SOLVE_MIXED_F32)
    xg = layout.from_full(layout.real_to_complex(xh).reshape(2, -1, 4, 3, Ls), L)
    assert krylov.true_residual(U, xg, b, M5, mf) <= 1e-9 * 1.01
    ctx.close()


def test_rbcg_zero_source_and_maxiter():
    L, Ls = (4, 4, 4, 4), 4
    U = synth.random_gauge(L, 0.3, 5)
    ctx = ops.Context(L, Ls, M5, U)
    z = ctx.new_full(F64)
    x = ctx.new_full(F64)
    st = ops.rbcg_solve(ctx, x, z, 0.01, 1e-8, 10, SOLVE_MIXED_F32)
    assert st["iterations"] == 0 and float(x.abs().max()) == 0.0
    b = full_dev(synth.gaussian_spinor(L, Ls, 6), L, F64)
    with pytest.raises(DWFError) as e:
        ops.rbcg_solve(ctx, x, b, 0.01, 1e-12, 3, SOLVE_MIXED_F32)
    assert e.value.code == -3
    ctx.close()


def test_bad_arguments_are_rejected(case):
    L, Ls, U, ctx = case
    a = ctx.new_half(F32)
    with pytest.raises(DWFError) as e:
        ops.dwf_dhop(ctx, a, a, 2)
    assert e.value.code == DWF_EINVAL
    with pytest.raises(DWFError):
        ops.dwf_mpc(ctx, a, a, 0.01)
    with pytest.raises(DWFError):
        ops.dwf_dhop(ctx, a, a, 0, nrhs=0)


def test_power_method(case):
    L, Ls, U, ctx = case
    mf = 0.05
    v0 = synth.gaussian_spinor(L, Ls, 17)
    got = ops.dwf_power_max(ctx, full_dev(v0, L, F64), mf, 30)
    want = krylov.power_max(lambda v: dwf.mdagm(U, v, M5, mf), v0, 30)
    assert got == pytest.approx(want, rel=1e-10)


def test_power_method_f32(case):
    """The FP32 power method (the option the multigrid setup uses to bound
    its filter interval) against the FP64 oracle's iteration from the same
    start: the power iteration contracts towards the top eigenvector, so the
    FP32 roundings of each step (relative 1e-7) do not accumulate, and the
    Rayleigh quotient is accurate to the FP32 operator bound."""
    L, Ls, U, ctx = case
    mf = 0.05
    v0 = synth.gaussian_spinor(L, Ls, 17)
    got = ops.dwf_power_max(ctx, full_dev(v0, L, F64), mf, 30, F32)
    want = krylov.power_max(lambda v: dwf.mdagm(U, v, M5, mf), v0, 30)
    print(f"power method F32: rel err {abs(got - want) / want:.3e}")
    assert got == pytest.approx(want, rel=1e-6)


@pytest.mark.parametrize("prec", [F32, F16S])
@pytest.mark.parametrize("variant", range(_lib.HOP_VARIANTS))
def test_every_hop_variant_matches_oracle(prec, variant):
    """Each tuning variant of the hopping kernel (register caps, prefetch,
    packed FP32 arithmetic, hypercube tiles, s-pairs, multi-row CTAs)
    reproduces the oracle, plain and with the fused M_ee / M_ee^-1 epilogues
    of M_pc."""
    from paper_2103_05034_gb300 import layout
    rows = 4 if variant in (16, 17) else 2 if variant in (14, 15) else 1  # CTAs over several y-rows
    cases = [((16, 4, 2, 2), 16), ((16, 4, 2, 2), 24)]  # x segments of 8 sites, 4 rows
    if rows == 1:
        cases += [((4, 4, 2, 2), 16), ((2, 4, 2, 2), 24)]
    for L, Ls in cases:
        U = synth.random_gauge(L, 0.5, 8)
        ctx = ops.Context(L, Ls, M5, U)
        ops.dwf_set_hop_variant(ctx, prec, variant)
        psi = synth.gaussian_spinor(L, Ls, 31)
        for dagger in (0, 1):
            inp = half_dev(psi, L, 1, prec)
            out = torch.zeros_like(inp)
            ops.dwf_dhop(ctx, out, inp, 0, dagger)
            want = layout.to_half(dwf.dhop(U, dwf.project_parity(psi, L, 1), dag=bool(dagger)), L, 0)
            assert rel(dev_to_half(out, Ls), want) < TOL[prec]
        if prec == F32:
            pe = dwf.project_parity(psi, L, 0)
            inp = half_dev(psi, L, 0, prec)
            out = torch.zeros_like(inp)
            ops.dwf_mpc(ctx, out, inp, 0.05, 1)
            assert rel(dev_to_half(out, Ls), layout.to_half(dwf.mpc_dag(U, pe, M5, 0.05), L, 0)) < TOL[prec]
        ctx.close()


def test_row_block_variant_rejected_where_it_does_not_tile():
    """A multi-row variant on a lattice whose x extent is not a multiple of
    the 8-site segment is refused (DWF_EINVAL), never launched."""
    L, Ls = (4, 4, 2, 2), 16
    ctx = ops.Context(L, Ls, M5, synth.random_gauge(L, 0.5, 8))
    with pytest.raises(DWFError) as e:
        ops.dwf_set_hop_variant(ctx, F32, 16)
    assert e.value.code == DWF_EINVAL
    ctx.close()


def test_bounded_waits_give_up_and_report():
    """Failure detection without a GPU fault: a poll on a counter and an
    mbarrier wait that nothing completes each give up after about a
    millisecond, the status reaches the host as DWF_ETIMEOUT, and the context
    keeps working afterwards."""
    import ctypes as C
    from paper_2103_05034_gb300._lib import DWF_ETIMEOUT
    gave_up = (C.c_int * 2)(-1, -1)
    code = _lib.lib().dwf_selftest_wait_timeout(gave_up, None)
    assert code == DWF_ETIMEOUT
    assert list(gave_up) == [1, 1]
    L, Ls = (4, 4, 2, 2), 8
    ctx = ops.Context(L, Ls, M5, synth.random_gauge(L, 0.5, 8))
    a = ctx.new_half(F32)
    a.fill_(1.0)
    assert ops.dwf_norm2(ctx, a) == pytest.approx(a.numel() / 2 * 2.0, rel=1e-6)
    ctx.close()


# ------------------------------------------------------------ float-float FP64 operator
# FP64 storage with float-float arithmetic (pairs of FP32 numbers with
# error-free sums and products, about 46 significant bits): a few dozen
# roundings of relative size 2^-46 ~ 1.4e-14 per output, so 1e-12 as for FP64.
@pytest.fixture
def df_mode(case):
    L, Ls, U, ctx = case
    ops.set_f64_arithmetic(ctx, _lib.ARITH_FLOAT_FLOAT)
    yield case
    ops.set_f64_arithmetic(ctx, _lib.ARITH_FP64)


@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_dhop_float_float(df_mode, dagger, out_parity):
    L, Ls, U, ctx = df_mode
    from paper_2103_05034_gb300 import layout
    psi = synth.gaussian_spinor(L, Ls, 11)
    src = dwf.project_parity(psi, L, 1 - out_parity)
    inp = half_dev(psi, L, 1 - out_parity, F64)
    out = torch.zeros_like(inp)
    ops.dwf_dhop(ctx, out, inp, out_parity, dagger)
    want = layout.to_half(dwf.dhop(U, src, dag=bool(dagger)), L, out_parity)
    got = dev_to_half(out, Ls)
    assert rel(got, want) < 1e-12
    # not the FP64 kernel: the result differs from it in the last bits
    ops.set_f64_arithmetic(ctx, _lib.ARITH_FP64)
    out64 = torch.zeros_like(inp)
    ops.dwf_dhop(ctx, out64, inp, out_parity, dagger)
    assert not torch.equal(out, out64)


def test_mpc_ddw_hdw_float_float(df_mode):
    """The fused epilogues (M_ee, M_ee^-1, Gamma_5) in float-float."""
    L, Ls, U, ctx = df_mode
    from paper_2103_05034_gb300 import layout
    mf = 0.05
    psi = dwf.project_parity(synth.gaussian_spinor(L, Ls, 13), L, 0)
    inp = half_dev(psi, L, 0, F64)
    out = torch.zeros_like(inp)
    for dagger, fn in ((0, dwf.mpc), (1, dwf.mpc_dag)):
        ops.dwf_mpc(ctx, out, inp, mf, dagger)
        assert rel(dev_to_half(out, Ls), layout.to_half(fn(U, psi, M5, mf), L, 0)) < 1e-12
    full = synth.gaussian_spinor(L, Ls, 14)
    fin = full_dev(full, L, F64)
    fout = torch.zeros_like(fin)
    ops.dwf_ddw(ctx, fout, fin, mf, 1)
    assert rel(dev_to_full_canon(fout, L, Ls), dwf.ddw(U, full, M5, mf, dag=True)) < 1e-12
    ops.dwf_hdw(ctx, fout, fin, mf)
    assert rel(dev_to_full_canon(fout, L, Ls), dwf.hdw(U, full, M5, mf)) < 1e-12


@pytest.mark.parametrize("policy", [SOLVE_F64, SOLVE_MIXED_F32])
def test_rbcg_float_float_operator(policy):
    """The red-black CG with the FP64 operator in float-float arithmetic
    (source preparation, reliable updates, reconstruction, true residual):
    the true residual reaches 1e-10 and the solution matches the oracle's."""
    L, Ls, mf = (4, 4, 4, 4), 8, 0.01
    U = synth.random_gauge(L, 0.3, synth.SEED_GAUGE)
    b = synth.gaussian_spinor(L, Ls, synth.SEED_SOURCE)
    ctx = ops.Context(L, Ls, M5, U)
    ops.set_f64_arithmetic(ctx, _lib.ARITH_FLOAT_FLOAT)
    tol = 1e-10
    bd = full_dev(b, L, F64)
    x = torch.zeros_like(bd)
    st = ops.rbcg_solve(ctx, x, bd, mf, tol, 20000, policy)
    xg = dev_to_full_canon(x, L, Ls)
    res = krylov.true_residual(U, xg, b, M5, mf)
    assert res <= tol * 1.01, st
    assert st["true_residual"] == pytest.approx(res, rel=1e-3, abs=1e-13)
    xr, _, _ = krylov.rbcg_solve(U, b, M5, mf, 1e-13)
    assert rel(xg, xr) < 1e-7
    ctx.close()


def test_float_float_small_and_large_values():
    """Inputs spanning many binades (1e-20 .. 1e20 times a Gaussian): the
    float-float hop keeps 1e-12 relative accuracy per output where the
    inputs are within the FP32 exponent range."""
    L, Ls = (4, 4, 2, 2), 16
    U = synth.random_gauge(L, 0.5, 9)
    ctx = ops.Context(L, Ls, M5, U)
    ops.set_f64_arithmetic(ctx, _lib.ARITH_FLOAT_FLOAT)
    from paper_2103_05034_gb300 import layout
    for scale in (1e-20, 1e-3, 1e8, 1e20):
        psi = scale * synth.gaussian_spinor(L, Ls, 17)
        src = dwf.project_parity(psi, L, 1)
        inp = half_dev(psi, L, 1, F64)
        out = torch.zeros_like(inp)
        ops.dwf_dhop(ctx, out, inp, 0, 0)
        want = layout.to_half(dwf.dhop(U, src), L, 0)
        assert rel(dev_to_half(out, Ls), want) < 1e-12, scale
    ctx.close()
