"""torch.autograd.Functions for the pseudofermion actions of the HMC in which
the paper's solvers run (Sec. 6 of arXiv:2103.05034), on the red-black
operator M = M_pc of Sec. 5.1:

  DWFPseudofermionAction  S   = sum_i phi_i^dag (M(m_i)^dag M(m_i))^-1 phi_i
  DWFRatioAction          S_r = sum_i phi_i^dag M(m2_i) (M(m1_i)^dag M(m1_i))^-1
                                M(m2_i)^dag phi_i   (Hasenbusch ratio factors)

forward: the normal-equation solves of all fields as one batched red-black CG
through the C ABI (rbcg_normal_solve_batch: each hopping launch covers every
field, each with its own mass; FP64 reliable updates), then the action by the
library's variational estimator (dwf_pf_action, error quadratic in the solve
residual).  backward: the hand-written force kernels (dwf_force,
dwf_ratio_force).  This module only moves tensors between those calls.

The gradient returned for the link field U is the Lie-algebra force G of the
convention dS/deps = sum Re tr(G^dag Q) for U -> exp(eps Q) U, Q in su(3): the
quantity an HMC integrator consumes.  For su(3) directions Q it equals the
directional derivative that torch's complex-gradient convention gives.
"""
from __future__ import annotations

import torch

from . import ops


class DWFPseudofermionAction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, U, ctx, phis, masses, tol=1e-12):
        """U: complex128 gauge tensor (only used to carry the gradient; the
        context `ctx` holds the same links).  phis: list of FP64 even half-field
        tensors (interleaved re, im).  Returns S (float64 scalar tensor)."""
        phi_all = torch.cat([p.reshape(-1) for p in phis])
        X_all = torch.zeros_like(phi_all)
        ops.rbcg_normal_solve_batch(ctx, X_all, phi_all, list(masses), tol)
        S = ops.dwf_pf_action(ctx, phi_all, X_all, list(masses))
        fctx.ctx = ctx
        fctx.masses = list(masses)
        fctx.save_for_backward(X_all)
        fctx.gshape = U.shape
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(fctx, grad_out):
        (X,) = fctx.saved_tensors
        G = torch.zeros(fctx.gshape, dtype=torch.complex128, device=X.device)
        ops.dwf_force(fctx.ctx, torch.view_as_real(G), X, fctx.masses)
        return G * grad_out, None, None, None, None


class DWFRatioAction(torch.autograd.Function):
    @staticmethod
    def forward(fctx, U, ctx, phis, m1, m2, tol=1e-12):
        """phis: list of FP64 even half fields, one per ratio factor, factor i
        with masses m1[i] (the inverted operator) and m2[i]."""
        phi_all = torch.cat([p.reshape(-1) for p in phis])
        chi = torch.zeros_like(phi_all)
        for i, m in enumerate(m2):  # chi_i = M(m2_i)^dag phi_i
            ops.dwf_mpc(ctx, chi.view(len(phis), -1)[i], phi_all.view(len(phis), -1)[i], m, dagger=1)
        X_all = torch.zeros_like(phi_all)
        ops.rbcg_normal_solve_batch(ctx, X_all, chi, list(m1), tol)
        S = ops.dwf_pf_action(ctx, chi, X_all, list(m1))
        fctx.ctx = ctx
        fctx.m1, fctx.m2 = list(m1), list(m2)
        fctx.save_for_backward(X_all, phi_all)
        fctx.gshape = U.shape
        return torch.tensor(S, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(fctx, grad_out):
        X, phi = fctx.saved_tensors
        G = torch.zeros(fctx.gshape, dtype=torch.complex128, device=X.device)
        ops.dwf_ratio_force(fctx.ctx, torch.view_as_real(G), X, phi, fctx.m1, fctx.m2)
        return G * grad_out, None, None, None, None, None


def pseudofermion_action(U, ctx, phis, masses, tol=1e-12):
    return DWFPseudofermionAction.apply(U, ctx, phis, masses, tol)


def ratio_action(U, ctx, phis, m1, m2, tol=1e-12):
    return DWFRatioAction.apply(U, ctx, phis, m1, m2, tol)
