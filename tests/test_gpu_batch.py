"""GPU parity of the batched red-black CG (rbcg_solve_batch,
rbcg_normal_solve_batch) through the C ABI: several right-hand sides, each
with its own mass, solved together (Sec. 5.1 operator; the pseudofermion
masses of the HMC setting of Sec. 6), against the FP64 oracle's per-mass
solves and against the single-rhs solver."""
import numpy as np
import pytest
import torch

import synth
from oracle import dwf, force, krylov
from paper_2103_05034_gb300 import layout, ops
from paper_2103_05034_gb300._lib import (DWF_EINVAL, F64, SOLVE_F64, SOLVE_MIXED_F16, SOLVE_MIXED_F32,
                                         DWFError)

from gpu_helpers import dev_to_full_canon, full_dev, half_dev, rel

pytestmark = pytest.mark.gpu
M5 = 1.8
HASENBUSCH = [0.01, 0.05, 0.2, 1.0]


def _batch_full(srcs, L):
    return torch.cat([full_dev(b, L, F64).reshape(-1) for b in srcs])


@pytest.mark.parametrize("policy", [SOLVE_F64, SOLVE_MIXED_F32])
def test_rbcg_batch_matches_oracle(policy):
    """4^4 x Ls=8, U = exp(0.3 i H): four sources with the masses 0.01, 0.05,
    0.2, 1.0 in one batch; every solution against the oracle's red-black CG
    for its own mass, and the true residuals recomputed by the oracle."""
    L, Ls, tol = (4, 4, 4, 4), 8, 1e-10
    U = synth.random_gauge(L, 0.3, synth.SEED_GAUGE)
    srcs = [synth.gaussian_spinor(L, Ls, 300 + i) for i in range(4)]
    ctx = ops.Context(L, Ls, M5, U)
    b = _batch_full(srcs, L)
    x = torch.zeros_like(b)
    st = ops.rbcg_solve_batch(ctx, x, b, HASENBUSCH, tol, 20000, policy)
    xs = x.view(4, -1)
    for i, (src, m) in enumerate(zip(srcs, HASENBUSCH)):
        xg = dev_to_full_canon(xs[i], L, Ls)
        res = krylov.true_residual(U, xg, src, M5, m)
        assert res <= tol * 1.01, (i, st[i])
        assert st[i]["true_residual"] == pytest.approx(res, rel=1e-3, abs=1e-14)
        xr, it, _ = krylov.rbcg_solve(U, src, M5, m, 1e-13)
        assert rel(xg, xr) < 1e-7
        if policy == SOLVE_F64:
            # each rhs runs its own CG recurrence: its iteration count is that
            # of the oracle's CG for the same mass, up to the check interval
            _, it10, _ = krylov.rbcg_solve(U, src, M5, m, tol)
            assert abs(st[i]["iterations"] - it10) <= 0.05 * it10 + 16, (i, st[i], it10)
    # the heavy mass converges first and stays put while the light ones continue
    assert st[3]["iterations"] < st[0]["iterations"]
    ctx.close()


def test_rbcg_batch_equals_single_solves():
    """4x4x4x8 x Ls=16 (several CTAs per launch), three masses: the batch
    against three single-rhs mixed-precision solves."""
    L, Ls, tol = (4, 4, 4, 8), 16, 1e-9
    masses = [0.02, 0.1, 0.5]
    U = synth.random_gauge(L, 0.5, 41, ape_steps=1)
    srcs = [synth.gaussian_spinor(L, Ls, 420 + i) for i in range(3)]
    ctx = ops.Context(L, Ls, M5, U)
    b = _batch_full(srcs, L)
    x = torch.zeros_like(b)
    st = ops.rbcg_solve_batch(ctx, x, b, masses, tol, 20000, SOLVE_MIXED_F32)
    xs = x.view(3, -1)
    bs = b.view(3, -1)
    for i, m in enumerate(masses):
        x1 = torch.zeros_like(bs[i])
        s1 = ops.rbcg_solve(ctx, x1, bs[i].clone(), m, tol, 20000, SOLVE_MIXED_F32)
        assert st[i]["true_residual"] <= tol and s1["true_residual"] <= tol
        a, c = xs[i].cpu().numpy(), x1.cpu().numpy()
        assert np.linalg.norm(a - c) / np.linalg.norm(c) < 1e-6
        # same recurrence per rhs: iteration counts close to the single solve's
        assert abs(st[i]["iterations"] - s1["iterations"]) <= 0.1 * s1["iterations"] + 16, (st[i], s1)
    ctx.close()


def test_rbcg_batch_single_rhs_and_host_buffers_with_zero_source():
    L, Ls, tol = (4, 4, 4, 4), 4, 1e-9
    U = synth.random_gauge(L, 0.3, 43)
    ctx = ops.Context(L, Ls, M5, U)
    src = synth.gaussian_spinor(L, Ls, 44)
    # nrhs = 1 agrees with the single-rhs solver
    b1 = full_dev(src, L, F64)
    xa, xb = torch.zeros_like(b1), torch.zeros_like(b1)
    sa = ops.rbcg_solve_batch(ctx, xa, b1, [0.05], tol, 5000, SOLVE_F64)[0]
    sb = ops.rbcg_solve(ctx, xb, b1, 0.05, tol, 5000, SOLVE_F64)
    assert sa["true_residual"] <= tol
    assert rel(xa.cpu().numpy(), xb.cpu().numpy()) < 1e-8
    assert abs(sa["iterations"] - sb["iterations"]) <= 8
    # host buffers, the middle source zero
    bh = np.concatenate([layout.complex_to_real(layout.to_full(src, L), F64),
                         np.zeros(layout.complex_to_real(layout.to_full(src, L), F64).shape),
                         layout.complex_to_real(layout.to_full(2.0 * src, L), F64)])
    xh = np.ones_like(bh)
    st = ops.rbcg_solve_batch(ctx, xh, bh, [0.05, 0.05, 0.3], tol, 5000, SOLVE_MIXED_F32)
    parts = xh.reshape(3, -1)
    assert not parts[1].any() and st[1]["iterations"] == 0 and st[1]["true_residual"] == 0.0
    for i, (s, m) in enumerate([(src, 0.05), (2.0 * src, 0.3)]):
        xg = layout.from_full(layout.real_to_complex(parts[2 * i]).reshape(2, -1, 4, 3, Ls), L)
        assert krylov.true_residual(U, xg, s, M5, m) <= tol * 1.01
    ctx.close()


def test_normal_solve_batch_matches_oracle():
    """The pseudofermion solves of the force workload's form (even parity,
    (M_pc^dag M_pc)^-1 phi) for the four masses in one batch."""
    L, Ls = (4, 4, 4, 4), 4
    U = synth.random_gauge(L, 0.5, 61)
    phis = [dwf.project_parity(synth.gaussian_spinor(L, Ls, 470 + i), L, 0) for i in range(4)]
    ctx = ops.Context(L, Ls, M5, U)
    pd = torch.cat([half_dev(p, L, 0, F64).reshape(-1) for p in phis])
    for policy in (SOLVE_F64, SOLVE_MIXED_F32):
        x = torch.zeros_like(pd)
        st = ops.rbcg_normal_solve_batch(ctx, x, pd, HASENBUSCH, 1e-12, 20000, policy)
        xs = x.view(4, -1)
        for i, (p, m) in enumerate(zip(phis, HASENBUSCH)):
            want = layout.to_half(force.solve_normal(U, p, M5, m), L, 0)
            got = layout.real_to_complex(xs[i].cpu().numpy()).reshape(want.shape)
            assert rel(got, want) < 1e-9, (i, st[i])
            assert st[i]["true_residual"] <= 1e-12
    ctx.close()


def test_batch_errors():
    L, Ls = (4, 4, 4, 4), 4
    U = synth.random_gauge(L, 0.3, 45)
    ctx = ops.Context(L, Ls, M5, U)
    src = synth.gaussian_spinor(L, Ls, 46)
    b = torch.cat([full_dev(src, L, F64).reshape(-1)] * 2)
    x = torch.zeros_like(b)
    for masses, policy in (([], SOLVE_F64), ([0.1] * 65, SOLVE_F64), ([0.1, float("nan")], SOLVE_F64),
                           ([0.1, 0.2], SOLVE_MIXED_F16)):
        with pytest.raises(DWFError) as e:
            ops.rbcg_solve_batch(ctx, x, b, masses, 1e-8, 100, policy)
        assert e.value.code == DWF_EINVAL
    with pytest.raises(DWFError) as e:
        ops.rbcg_solve_batch(ctx, x.cpu().numpy(), b, [0.1, 0.2], 1e-8, 100, SOLVE_F64)
    assert e.value.code == DWF_EINVAL
    ph = ctx.new_half(F64, nrhs=2)
    with pytest.raises(DWFError) as e:
        ops.rbcg_normal_solve_batch(ctx, ph, ph, [0.1, 0.2], 1e-8, 100, SOLVE_F64)
    assert e.value.code == DWF_EINVAL
    # maxiter reached: DWF_ENOCONV, with the iterate still written
    with pytest.raises(DWFError) as e:
        ops.rbcg_solve_batch(ctx, x, b, [0.01, 0.02], 1e-12, 3, SOLVE_MIXED_F32)
    assert e.value.code == -3
    assert float(x.abs().max()) > 0.0
    ctx.close()
