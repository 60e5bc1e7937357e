"""GPU parity of the pseudofermion force (dwf_force) and the autograd Function
against the FP64 oracle force, whose sign and normalisation are pinned by
finite differences (tests/test_oracle_mg.py)."""
import numpy as np
import pytest
import torch

import synth
from oracle import dwf, force
from paper_2103_05034_gb300 import autograd, layout, ops
from paper_2103_05034_gb300._lib import F32, F64, SOLVE_F64

from gpu_helpers import half_dev, rel

pytestmark = pytest.mark.gpu
M5 = 1.8


@pytest.fixture(scope="module")
def fcase():
    L, Ls = (4, 4, 4, 4), 4
    U = synth.random_gauge(L, 0.5, 61)
    masses = [0.05, 0.3]
    phis = [dwf.project_parity(synth.gaussian_spinor(L, Ls, 70 + i), L, 0) for i in range(2)]
    ctx = ops.Context(L, Ls, M5, U)
    G = force.force(U, phis, masses, M5)
    yield L, Ls, U, masses, phis, ctx, G
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(F64, 1e-11), (F32, 2e-5)])
def test_force_kernel_matches_oracle(fcase, prec, tol):
    L, Ls, U, masses, phis, ctx, G = fcase
    Xs = [force.solve_normal(U, p, M5, m) for p, m in zip(phis, masses)]
    Xd = torch.cat([half_dev(x, L, 0, prec).reshape(-1) for x in Xs])
    out = torch.zeros(U.shape, dtype=torch.complex128, device="cuda")
    ops.dwf_force(ctx, torch.view_as_real(out), Xd, masses)
    assert rel(out.cpu().numpy(), G) < tol


def test_normal_solve(fcase):
    L, Ls, U, masses, phis, ctx, G = fcase
    for p, m in zip(phis, masses):
        pd = half_dev(p, L, 0, F64)
        x = torch.zeros_like(pd)
        st = ops.rbcg_normal_solve(ctx, x, pd, m, 1e-12)
        want = layout.to_half(force.solve_normal(U, p, M5, m), L, 0)
        got = layout.real_to_complex(x.cpu().numpy()).reshape(want.shape)
        assert rel(got, want) < 1e-9, st
        assert st["true_residual"] <= 1e-12


def test_autograd_action_and_force(fcase):
    L, Ls, U, masses, phis, ctx, G = fcase
    Ut = torch.from_numpy(U).to("cuda").requires_grad_(True)
    pds = [half_dev(p, L, 0, F64) for p in phis]
    S = autograd.pseudofermion_action(Ut, ctx, pds, masses, 1e-12)
    S_or = force.action(U, phis, masses, M5)
    assert float(S) == pytest.approx(S_or, rel=1e-10)
    S.backward()
    assert rel(Ut.grad.cpu().numpy(), G) < 1e-8


def test_force_finite_difference_on_gpu(fcase):
    """Central differences of the GPU action along a random su(3) field Q
    (links exp(+-eps Q) U set up on the host) against sum Re tr(G^dag Q)."""
    L, Ls, U, masses, phis, ctx, G = fcase
    Q = synth.random_su3_algebra(U.shape[:-2], 83)
    eps = 1e-5
    pds = [half_dev(p, L, 0, F64) for p in phis]

    def S_of(links):
        c2 = ops.Context(L, Ls, M5, links)
        Ut = torch.from_numpy(links).to("cuda")
        s = float(autograd.pseudofermion_action(Ut, c2, pds, masses, 1e-13))
        c2.close()
        return s

    Up = np.einsum("...ij,...jk->...ik", force.exp_su3(eps * Q), U)
    Um = np.einsum("...ij,...jk->...ik", force.exp_su3(-eps * Q), U)
    fd = (S_of(Up) - S_of(Um)) / (2 * eps)
    an = np.sum(np.trace(np.conj(np.swapaxes(G, -1, -2)) @ Q, axis1=-2, axis2=-1)).real
    assert abs(fd - an) <= 1e-6 * abs(an)


# The force workload's shape: Ls = 16 and 24 (the k_force<P, 16, 8> and
# <P, 24, 8> CTA shapes), four pseudofermions at the Hasenbusch-style masses.
# The kernel takes X itself, so X is a Gaussian even field here (no solve):
# the oracle forms Y = M_pc X, the full fields X', Y' and G for each mass.
FORCE_MASSES = [0.01, 0.05, 0.2, 1.0]


@pytest.mark.parametrize("Ls", [16, 24])
@pytest.mark.parametrize("prec,tol", [(F64, 1e-11), (F32, 1e-5)])
def test_force_four_pseudofermions_at_ls16_ls24(Ls, prec, tol):
    """FP32 bound: the force is a sum over 4 directions x Ls slices x 4
    pseudofermions of O(1) outer products in FP32 (relative rounding ~6e-8 per
    term, summed over ~10^2 terms per site, plus the FP32 hops forming Y, X',
    Y'), well inside 1e-5 norm-wise."""
    L = (8, 4, 4, 4)
    U = synth.random_gauge(L, 0.5, 62, ape_steps=1)
    ctx = ops.Context(L, Ls, M5, U)
    Xs = [dwf.project_parity(synth.gaussian_spinor(L, Ls, 80 + i), L, 0) for i in range(4)]
    G = np.zeros_like(U)
    for X, m in zip(Xs, FORCE_MASSES):
        Y = dwf.mpc(U, X, M5, m)
        Xf, Yf = force.bilinear_fields(U, X, Y, M5, m)
        G += force.force_from_fields(U, Xf, Yf)
    Xd = torch.cat([half_dev(x, L, 0, prec).reshape(-1) for x in Xs])
    out = torch.zeros(U.shape, dtype=torch.complex128, device="cuda")
    ops.dwf_force(ctx, torch.view_as_real(out), Xd, FORCE_MASSES)
    assert rel(out.cpu().numpy(), G) < tol
    ctx.close()


# ---------------------------------------------------------------- Hasenbusch ratio factors
def _ratio_oracle_from_fields(U, X, phi, m1, m2):
    """G_r for given X and phi (no solve): G(X', (M1 X)'; m1) - G(X', phi'; m2)."""
    Y = dwf.mpc(U, X, M5, m1)
    Xf1, Yf1 = force.bilinear_fields(U, X, Y, M5, m1)
    Xf2, Pf2 = force.bilinear_fields(U, X, phi, M5, m2)
    return force.force_from_fields(U, Xf1, Yf1) - force.force_from_fields(U, Xf2, Pf2)


@pytest.mark.parametrize("prec,tol", [(F64, 1e-11), (F32, 1e-5)])
def test_ratio_force_kernel_matches_oracle(prec, tol):
    L, Ls = (4, 4, 4, 4), 8
    U = synth.random_gauge(L, 0.5, 63)
    ctx = ops.Context(L, Ls, M5, U)
    m1, m2 = [0.01, 0.2], [0.05, 1.0]
    Xs = [dwf.project_parity(synth.gaussian_spinor(L, Ls, 90 + i), L, 0) for i in range(2)]
    Ps = [dwf.project_parity(synth.gaussian_spinor(L, Ls, 95 + i), L, 0) for i in range(2)]
    G = sum(_ratio_oracle_from_fields(U, X, P, a, b) for X, P, a, b in zip(Xs, Ps, m1, m2))
    Xd = torch.cat([half_dev(x, L, 0, prec).reshape(-1) for x in Xs])
    Pd = torch.cat([half_dev(p, L, 0, prec).reshape(-1) for p in Ps])
    out = torch.zeros(U.shape, dtype=torch.complex128, device="cuda")
    ops.dwf_ratio_force(ctx, torch.view_as_real(out), Xd, Pd, m1, m2)
    assert rel(out.cpu().numpy(), G) < tol
    ctx.close()


@pytest.fixture(scope="module")
def rcase():
    L, Ls = (4, 4, 4, 4), 4
    U = synth.random_gauge(L, 0.5, 64)
    ctx = ops.Context(L, Ls, M5, U)
    phi = dwf.project_parity(synth.gaussian_spinor(L, Ls, 97), L, 0)
    yield L, Ls, U, ctx, phi
    ctx.close()


def test_ratio_action_and_force_autograd(rcase):
    """S_r and its gradient through DWFRatioAction against the oracle's
    ratio_action and ratio_force (which solve (M1^dag M1) X = M2^dag phi
    themselves)."""
    L, Ls, U, ctx, phi = rcase
    m1, m2 = 0.02, 0.3
    Ut = torch.from_numpy(U).to("cuda").requires_grad_(True)
    S = autograd.ratio_action(Ut, ctx, [half_dev(phi, L, 0, F64)], [m1], [m2], 1e-12)
    assert float(S) == pytest.approx(force.ratio_action(U, phi, m1, m2, M5), rel=1e-10)
    S.backward()
    assert rel(Ut.grad.cpu().numpy(), force.ratio_force(U, phi, m1, m2, M5)) < 1e-8


def test_ratio_force_vanishes_for_equal_masses(rcase):
    """m1 = m2: S_r = phi^dag phi does not depend on U, and the two bilinears
    cancel: G_r is zero up to rounding of the O(|G|) terms."""
    L, Ls, U, ctx, phi = rcase
    m = 0.1
    Ut = torch.from_numpy(U).to("cuda").requires_grad_(True)
    pd = half_dev(phi, L, 0, F64)
    S = autograd.ratio_action(Ut, ctx, [pd], [m], [m], 1e-12)
    assert float(S) == pytest.approx(dwf.norm2(phi), rel=1e-10)
    S.backward()
    one = torch.zeros(U.shape, dtype=torch.complex128, device="cuda")
    X = torch.zeros_like(pd)
    ops.rbcg_normal_solve(ctx, X, pd, m, 1e-12)
    ops.dwf_force(ctx, torch.view_as_real(one), X, [m])  # the size of one bilinear's force
    assert float(Ut.grad.abs().max()) <= 1e-9 * float(one.abs().max())


def test_ratio_force_finite_difference_on_gpu(rcase):
    L, Ls, U, ctx, phi = rcase
    m1, m2 = 0.02, 0.3
    Q = synth.random_su3_algebra(U.shape[:-2], 84)
    eps = 1e-5
    pd = half_dev(phi, L, 0, F64)

    def S_of(links):
        c2 = ops.Context(L, Ls, M5, links)
        s = float(autograd.ratio_action(torch.from_numpy(links).to("cuda"), c2, [pd], [m1], [m2], 1e-13))
        c2.close()
        return s

    Up = np.einsum("...ij,...jk->...ik", force.exp_su3(eps * Q), U)
    Um = np.einsum("...ij,...jk->...ik", force.exp_su3(-eps * Q), U)
    fd = (S_of(Up) - S_of(Um)) / (2 * eps)
    Ut = torch.from_numpy(U).to("cuda").requires_grad_(True)
    autograd.ratio_action(Ut, ctx, [pd], [m1], [m2], 1e-13).backward()
    G = Ut.grad.cpu().numpy()
    an = np.sum(np.trace(np.conj(np.swapaxes(G, -1, -2)) @ Q, axis1=-2, axis2=-1)).real
    assert abs(fd - an) <= 1e-6 * abs(an)


# ---------------------------------------------------------------- the force workload at full size
def test_force_16x16x16x32_ls16_by_tiling():
    """dwf_force at the force workload's size (16^3 x 32, Ls = 16, four
    pseudofermions at the Hasenbusch-style masses) in FP64 and FP32: links and
    X are an 8^4 field tiled 2 x 2 x 2 x 4 (an even period, so parities are
    kept), whose force is the tiled force of the small field; every link of
    the GPU result is compared with the oracle's small-lattice force."""
    Lb, Ls = (8, 8, 8, 8), 16
    reps = (4, 2, 2, 2, 1, 1, 1)  # numpy order (T, Z, Y, X, ...)
    L = (16, 16, 16, 32)
    Ub = synth.random_gauge(Lb, 0.5, synth.SEED_GAUGE, ape_steps=3)
    Xb = [dwf.project_parity(synth.gaussian_spinor(Lb, Ls, 120 + i), Lb, 0) for i in range(4)]
    Gb = np.zeros_like(Ub)
    for X, m in zip(Xb, FORCE_MASSES):
        Xf, Yf = force.bilinear_fields(Ub, X, dwf.mpc(Ub, X, M5, m), M5, m)
        Gb += force.force_from_fields(Ub, Xf, Yf)
    want = np.tile(Gb, reps)
    ctx = ops.Context(L, Ls, M5, np.tile(Ub, reps))
    for prec, tol in ((F64, 1e-11), (F32, 1e-5)):
        Xd = torch.cat([half_dev(np.tile(x, reps), L, 0, prec).reshape(-1)
                        for x in Xb])
        out = torch.zeros(want.shape, dtype=torch.complex128, device="cuda")
        ops.dwf_force(ctx, torch.view_as_real(out), Xd, FORCE_MASSES)
        err = rel(out.cpu().numpy(), want)
        print(f"force 16^3x32 Ls16 prec={prec}: rel err {err:.3e}")
        assert err < tol
    ctx.close()


def test_force_finite_differences_20_directions_16x16x16x32():
    """The force workload's check: S = sum_i phi_i^dag (M^dag M)^-1 phi_i on
    the 16^3 x 32, Ls = 16 smeared-random links with four pseudofermions at
    masses 0.01, 0.05, 0.2, 1.0; the autograd gradient (dwf_force on the
    mixed-precision solutions) against FP64 central differences
    (S(e^{eps Q} U) - S(e^{-eps Q} U)) / 2 eps, eps = 1e-5, of the GPU action
    along 20 random su(3) fields Q, each normalised to unit norm: agreement
    within 1e-4 relative to max |dS/deps| over the directions (c10's bound; a
    direction whose derivative happens to be near zero is judged on the
    scale of the others)."""
    name = "dwf_16x16x16x32_ls16"
    w = synth.WORKLOADS[name]
    L, Ls = w["L"], w["Ls"]
    U = synth.workload_gauge(name)
    ctx = ops.Context(L, Ls, M5, U)
    gen = torch.Generator(device="cuda").manual_seed(synth.SEED_SOURCE + 5)
    nh = ctx.half_numel()
    phis = [torch.randn(nh, generator=gen, device="cuda", dtype=torch.float64) for _ in range(4)]
    Ut = torch.from_numpy(U).to("cuda").requires_grad_(True)
    autograd.pseudofermion_action(Ut, ctx, phis, FORCE_MASSES, 1e-12).backward()
    G = Ut.grad
    ctx.close()
    eps = 1e-5
    fds, ans = [], []
    for k in range(20):
        Q = synth.random_su3_algebra(U.shape[:-2], 1000 + k)
        Q /= np.sqrt(np.sum(np.abs(Q) ** 2))
        Qd = torch.from_numpy(Q).to("cuda")
        ans.append(float(torch.einsum("...ij,...ij->", torch.conj(G), Qd).real))  # sum Re tr(G^dag Q)
        vals = []
        for sgn in (1, -1):
            Ux = np.einsum("...ij,...jk->...ik", force.exp_su3(sgn * eps * Q), U)
            c2 = ops.Context(L, Ls, M5, Ux)
            vals.append(float(autograd.pseudofermion_action(torch.from_numpy(Ux).to("cuda"), c2, phis,
                                                              FORCE_MASSES, 1e-12)))
            c2.close()
        fds.append((vals[0] - vals[1]) / (2 * eps))
    fds, ans = np.array(fds), np.array(ans)
    scale = np.max(np.abs(ans))
    print("force FD 16^3: max |fd - G.Q| / max|G.Q| =", np.max(np.abs(fds - ans)) / scale)
    assert np.max(np.abs(fds - ans)) <= 1e-4 * scale
