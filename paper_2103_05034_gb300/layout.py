"""Host-side layout marshalling between canonical arrays and the library's
device field layout (include/dwfmg.h).

canonical spinor : complex (T, Z, Y, X, Ls, 4, 3)
device half field: complex (Vh, 4, 3, Ls) of one parity, sites in
                   lexicographic order (checkerboard index = lex // 2)
device full field: complex (2, Vh, 4, 3, Ls), even parity first
"""
from __future__ import annotations

import numpy as np


def parity_of_lex(L):
    Lx, Ly, Lz, Lt = L
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    return ((x + y + z + t) % 2).ravel()


def to_half(psi, L, parity):
    """Canonical (..., T, Z, Y, X, Ls, 4, 3) -> (..., Vh, 4, 3, Ls) of one parity."""
    lead = psi.shape[:-7]
    Ls = psi.shape[-3]
    v = psi.reshape(lead + (-1, Ls, 4, 3))
    sel = parity_of_lex(L) == parity
    v = v[..., sel, :, :, :]
    return np.ascontiguousarray(np.moveaxis(v, -3, -1))


def to_full(psi, L):
    """Canonical -> (..., 2, Vh, 4, 3, Ls)."""
    return np.stack([to_half(psi, L, 0), to_half(psi, L, 1)], axis=-5)


def from_half(h, L, parity, fill=None):
    """(..., Vh, 4, 3, Ls) -> canonical (..., T, Z, Y, X, Ls, 4, 3), zero elsewhere
    (or added into `fill`)."""
    Lx, Ly, Lz, Lt = L
    lead = h.shape[:-4]
    Ls = h.shape[-1]
    v = np.moveaxis(h, -1, -3)
    out = np.zeros(lead + (Lx * Ly * Lz * Lt, Ls, 4, 3), dtype=h.dtype) if fill is None else \
        fill.reshape(lead + (Lx * Ly * Lz * Lt, Ls, 4, 3))
    out[..., parity_of_lex(L) == parity, :, :, :] = v
    return out.reshape(lead + (Lt, Lz, Ly, Lx, Ls, 4, 3))


def from_full(f, L):
    out = from_half(f[..., 0, :, :, :, :], L, 0)
    return from_half(f[..., 1, :, :, :, :], L, 1, fill=out)


def complex_to_real(a, prec):
    """complex128 array -> interleaved real array of the storage precision."""
    dt = {0: np.float64, 1: np.float32, 2: np.float16}[prec]
    return np.ascontiguousarray(a).view(np.float64).astype(dt)


def real_to_complex(r):
    r = np.asarray(r, dtype=np.float64)
    return r.view(np.complex128)
