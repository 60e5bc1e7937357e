"""Parity at the paper's physical-point size, 48^3 x 96 x Ls=24, in the
launch configuration the benchmark times (autotuned FP32 hopping kernel).

The oracle cannot hold a 48^3 x 96 x 24 field, so the test uses translation
invariance: links and source are an 8^3 x 16 field tiled 6 x 6 x 6 x 6 (the
period is even, so parities are preserved).  D_hop of a tiled field is the
tiled D_hop of the small field, so every sampled output site of the GPU result
must equal the oracle's 8^3 x 16 result at the site modulo the period."""
import numpy as np
import pytest
import torch

import synth
from oracle import dwf
from paper_2103_05034_gb300 import layout, ops
from paper_2103_05034_gb300._lib import F32

pytestmark = pytest.mark.gpu


def test_dhop_48x48x48x96_ls24_by_tiling():
    Lb, Ls, tile = (8, 8, 8, 16), 24, 6
    L = tuple(l * tile for l in Lb)
    Ub = synth.random_gauge(Lb, 0.5, synth.SEED_GAUGE, ape_steps=3)
    psib = synth.gaussian_spinor(Lb, Ls, synth.SEED_SOURCE)
    want_b = dwf.dhop(Ub, dwf.project_parity(psib, Lb, 1))  # even output sites of the small field
    ctx = ops.Context(L, Ls, 1.8, np.tile(Ub, (tile, tile, tile, tile, 1, 1, 1)))
    ops.dwf_autotune(ctx, F32, 5)
    # tiled odd-parity source in the device layout, built on the GPU
    src = torch.from_numpy(psib.astype(np.complex64)).cuda().repeat(tile, tile, tile, tile, 1, 1, 1)
    par = torch.from_numpy(layout.parity_of_lex(L)).cuda()
    odd = src.reshape(-1, Ls, 4, 3)[par == 1].permute(0, 2, 3, 1).contiguous()
    del src
    inp = torch.view_as_real(odd).reshape(-1)
    out = torch.zeros_like(inp)
    ops.dwf_dhop(ctx, out, inp, 0)
    got = torch.view_as_complex(out.reshape(-1, 4, 3, Ls, 2))
    rng = np.random.default_rng(5)
    Vh = int(np.prod(L)) // 2
    hs = rng.integers(0, Vh, 2000)
    Lx, Ly, Lz, Lt = L
    xh = hs % (Lx // 2)
    rem = hs // (Lx // 2)
    y, z, t = rem % Ly, (rem // Ly) % Lz, rem // (Ly * Lz)
    x = 2 * xh + ((y + z + t) & 1)
    g = got[torch.from_numpy(hs).cuda()].cpu().numpy().astype(np.complex128)  # (n, 4, 3, Ls)
    w = want_b[t % Lb[3], z % Lb[2], y % Lb[1], x % Lb[0]]  # (n, Ls, 4, 3)
    w = np.moveaxis(w, 1, 3)
    assert np.linalg.norm(g - w) / np.linalg.norm(w) < 1e-6
    ctx.close()
