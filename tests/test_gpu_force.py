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
