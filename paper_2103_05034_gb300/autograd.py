"""torch.autograd.Function for the pseudofermion action
S = sum_i phi_i^dag (M_pc(m_i)^dag M_pc(m_i))^-1 phi_i
(red-black operator of Sec. 5.1 of arXiv:2103.05034; HMC context, Sec. 6).

forward: the normal-equation solves of all pseudofermions as one batched
red-black CG through the C ABI (rbcg_normal_solve_batch: each hopping launch
covers every pseudofermion, each with its own mass; FP64 reliable updates), S
evaluated with the estimator 2 Re<phi, X> - <X, M^dag M X> whose error is
quadratic in the solve residual.  backward: the hand-written force kernel
(dwf_force).

The gradient returned for the link field U is the Lie-algebra force G of the
convention dS/deps = sum Re tr(G^dag Q) for U -> exp(eps Q) U, Q in su(3): the
quantity an HMC integrator consumes.  For su(3) directions Q it equals the
directional derivative that torch's complex-gradient convention gives.
"""
from __future__ import annotations

import torch

from . import ops
from ._lib import F64, SOLVE_MIXED_F32


class DWFPseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, U, ctx, phis, masses, tol=1e-12):
        """U: complex128 gauge tensor (only used to carry the gradient; the
        context `ctx` holds the same links).  phis: list of FP64 even half-field
        tensors (interleaved re, im).  Returns S (float64 scalar tensor)."""
        phi_all = torch.cat([p.reshape(-1) for p in phis])
        X_all = torch.zeros_like(phi_all)
        ops.rbcg_normal_solve_batch(ctx, X_all, phi_all, list(masses), tol)
        Xs = list(X_all.view(len(phis), -1).unbind(0))
        S = 0.0
        for phi, X, mf in zip(phis, Xs, masses):
            X = X.view_as(phi)
            MX = torch.zeros_like(phi)
            ops.dwf_mpcdag_mpc(ctx, MX, X, mf)
            S += 2.0 * ops.dwf_cdot(ctx, phi, X).real - ops.dwf_cdot(ctx, X, MX).real
        fctx.ctx = ctx
        fctx.masses = list(masses)
        fctx.save_for_backward(X_all)
        fctx.gshape = U.shape
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(fctx, grad_out):
        (X,) = fctx.saved_tensors
        G = torch.zeros(fctx.gshape, dtype=torch.complex128, device=X.device)
        Gr = torch.view_as_real(G)
        ops.dwf_force(fctx.ctx, Gr, X, fctx.masses)
        return G * grad_out, None, None, None, None


def pseudofermion_action(U, ctx, phis, masses, tol=1e-12):
    return DWFPseudofermionAction.apply(U, ctx, phis, masses, tol)
