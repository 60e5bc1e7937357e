"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds no arithmetic of the multigrid method itself: it only draws
random numbers and builds stand-in gauge fields and sources with the shape and
statistics of the paper's workloads (Section 5: 16^3x32 and 48^3x96 lattices,
Ls = 16 / 24).  The real RBC/UKQCD configurations are not available, so
smeared-random SU(3) fields stand in for them.

Random numbers come from one counter-based generator: SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) as
a hash of (seed, counter), 53-bit uniforms, and the Box-Muller transform.  It
is written with vectorised numpy uint64 arithmetic, so the same seed gives the
same bits on x86_64 and aarch64 and for any numpy version.

Array conventions (canonical, host side):
  links   : complex128 (T, Z, Y, X, 4, 3, 3), mu = 0..3 is x, y, z, t,
            U_mu(x) is the parallel transporter from x to x + mu.
  spinors : complex128 (T, Z, Y, X, Ls, 4, 3).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (finaliser) on a uint64 array."""
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in (0, 1): element i is the (offset+i+1)-th SplitMix64 output
    of a generator seeded with `seed`."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN
        bits = _mix64(state)
    return ((bits >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal deviates by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    th = 2.0 * np.pi * u[1::2]
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    return out[:n]


def complex_gaussian(seed: int, shape) -> np.ndarray:
    """Complex Gaussian array, unit variance for each real component."""
    n = int(np.prod(shape))
    g = normal(seed, 2 * n)
    return (g[0::2] + 1j * g[1::2]).reshape(shape)


def spinor_shape(L, Ls):
    Lx, Ly, Lz, Lt = L
    return (Lt, Lz, Ly, Lx, Ls, 4, 3)


def gaussian_spinor(L, Ls, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Gaussian 5D source(s); with nrhs, shape (nrhs, T, Z, Y, X, Ls, 4, 3)."""
    shp = spinor_shape(L, Ls)
    if nrhs is None:
        return complex_gaussian(seed, shp)
    return complex_gaussian(seed, (nrhs,) + shp)


# Gell-Mann matrices lambda_1..lambda_8 (tr(l_a l_b) = 2 delta_ab).
_GM = np.zeros((8, 3, 3), dtype=complex)
_GM[0][0, 1] = _GM[0][1, 0] = 1
_GM[1][0, 1], _GM[1][1, 0] = -1j, 1j
_GM[2][0, 0], _GM[2][1, 1] = 1, -1
_GM[3][0, 2] = _GM[3][2, 0] = 1
_GM[4][0, 2], _GM[4][2, 0] = -1j, 1j
_GM[5][1, 2] = _GM[5][2, 1] = 1
_GM[6][1, 2], _GM[6][2, 1] = -1j, 1j
_GM[7] = np.diag([1, 1, -2]) / np.sqrt(3)


def _expi_hermitian(H: np.ndarray, eps: float) -> np.ndarray:
    """exp(i eps H) for a batch of 3x3 hermitian H by eigendecomposition."""
    w, V = np.linalg.eigh(H)
    return np.einsum("...ij,...j,...kj->...ik", V, np.exp(1j * eps * w), V.conj())


def project_su3(V: np.ndarray) -> np.ndarray:
    """Nearest unitary matrix W = V (V^dag V)^(-1/2) (polar decomposition),
    then the determinant phase removed with the principal cube root."""
    VdV = np.einsum("...ji,...jk->...ik", V.conj(), V)
    w, E = np.linalg.eigh(VdV)
    inv_sqrt = np.einsum("...ij,...j,...kj->...ik", E, 1.0 / np.sqrt(w), E.conj())
    W = V @ inv_sqrt
    det = np.linalg.det(W)
    return W / (det ** (1.0 / 3.0))[..., None, None]


_AX = (3, 2, 1, 0)  # array axis of direction mu in a (T, Z, Y, X, ...) array


def _shift(f, mu, sign):
    """f(x + sign*mu) as a field at x (periodic)."""
    return np.roll(f, -sign, axis=_AX[mu])


def ape_step(U: np.ndarray, alpha: float) -> np.ndarray:
    """One APE-style step: V = (1-alpha) U + (alpha/6) sum of the six staples,
    projected back to SU(3)."""
    Ud = lambda A: np.conj(np.swapaxes(A, -1, -2))
    new = np.empty_like(U)
    for mu in range(4):
        st = np.zeros(U.shape[:4] + (3, 3), dtype=complex)
        Umu = U[..., mu, :, :]
        for nu in range(4):
            if nu == mu:
                continue
            Unu = U[..., nu, :, :]
            # x -> x+nu -> x+nu+mu -> x+mu
            st += Unu @ _shift(Umu, nu, +1) @ Ud(_shift(Unu, mu, +1))
            # x -> x-nu -> x-nu+mu -> x+mu
            Unu_m = _shift(Unu, nu, -1)
            st += Ud(Unu_m) @ _shift(Umu, nu, -1) @ _shift(_shift(Unu, nu, -1), mu, +1)
        new[..., mu, :, :] = project_su3((1.0 - alpha) * Umu + (alpha / 6.0) * st)
    return new


def random_gauge(L, eps: float, seed: int, ape_steps: int = 0, alpha: float = 0.5) -> np.ndarray:
    """U_mu(x) = exp(i eps H), H = sum_a w_a lambda_a / 2 with w_a ~ N(0,1),
    followed by `ape_steps` APE-style smearing steps."""
    Lx, Ly, Lz, Lt = L
    shp = (Lt, Lz, Ly, Lx, 4)
    w = normal(seed, int(np.prod(shp)) * 8).reshape(shp + (8,))
    H = 0.5 * np.einsum("...a,aij->...ij", w, _GM)
    U = _expi_hermitian(H, eps)
    for _ in range(ape_steps):
        U = ape_step(U, alpha)
    return U


def random_gauge_transform(L, seed: int) -> np.ndarray:
    """Random SU(3) matrix per 4D site, shape (T, Z, Y, X, 3, 3)."""
    Lx, Ly, Lz, Lt = L
    shp = (Lt, Lz, Ly, Lx)
    w = normal(seed, int(np.prod(shp)) * 8).reshape(shp + (8,))
    H = 0.5 * np.einsum("...a,aij->...ij", w, _GM)
    return _expi_hermitian(H, 1.0)


def random_su3_algebra(shape, seed: int) -> np.ndarray:
    """Random traceless anti-hermitian 3x3 matrices Q = i sum_a w_a lambda_a/2."""
    n = int(np.prod(shape))
    w = normal(seed, n * 8).reshape(tuple(shape) + (8,))
    return 1j * 0.5 * np.einsum("...a,aij->...ij", w, _GM)


# Workload recipes (paper Section 5 shapes; synthetic smeared-random fields).
WORKLOADS = {
    # 4^4 x Ls=8, eps 0.3, no smearing, FP64: small parity case
    "dwf_4x4x4x4_ls8": dict(L=(4, 4, 4, 4), Ls=8, eps=0.3, ape=0, M5=1.8, mf=0.01),
    # 16^3 x 32 x Ls=16, eps 0.5, 3 APE steps: the paper's 16^3 test volume
    "dwf_16x16x16x32_ls16": dict(L=(16, 16, 16, 32), Ls=16, eps=0.5, ape=3, M5=1.8, mf=0.01),
    # 48^3 x 96 x Ls=24: the paper's physical-point volume.  Its links are the
    # 16^3 x 32 smeared field tiled 3 x 3 x 3 x 3 (still an SU(3) field, same
    # local statistics; generating 42M smeared links on the host is too slow)
    "dwf_48x48x48x96_ls24": dict(L=(48, 48, 48, 96), Ls=24, eps=0.5, ape=3, M5=1.8, mf=0.00078,
                                 tile_of="dwf_16x16x16x32_ls16", tile=(3, 3, 3, 3)),
    # the largest volume on which the multigrid with 32 FP32 basis vectors fits
    # one GPU (Ls = 24 and the mass of the physical-point workload); links: a
    # smeared 8^3 x 16 field tiled 3 x 3 x 3 x 3
    "dwf_24x24x24x48_ls24": dict(L=(24, 24, 24, 48), Ls=24, eps=0.5, ape=3, M5=1.8, mf=0.00078,
                                 tile_of="dwf_8x8x8x16_ls24", tile=(3, 3, 3, 3)),
    "dwf_8x8x8x16_ls24": dict(L=(8, 8, 8, 16), Ls=24, eps=0.5, ape=3, M5=1.8, mf=0.00078),
    # an intermediate Ls = 24 volume for profiling (links: the 16^3 x 32 field tiled twice)
    "dwf_32x32x32x64_ls24": dict(L=(32, 32, 32, 64), Ls=24, eps=0.5, ape=3, M5=1.8, mf=0.00078,
                                 tile_of="dwf_16x16x16x32_ls16", tile=(2, 2, 2, 2)),
}


def workload_gauge(name: str) -> np.ndarray:
    """The link field of a named workload (generated, or tiled from a smaller one)."""
    w = WORKLOADS[name]
    if "tile_of" in w:
        base = WORKLOADS[w["tile_of"]]
        U = random_gauge(base["L"], base["eps"], SEED_GAUGE, ape_steps=base["ape"])
        tx, ty, tz, tt = w["tile"]
        return np.tile(U, (tt, tz, ty, tx, 1, 1, 1))
    return random_gauge(w["L"], w["eps"], SEED_GAUGE, ape_steps=w["ape"])

SEED_GAUGE = 2103
SEED_SOURCE = 5034
SEED_BASIS = 1
