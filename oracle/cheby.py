"""Chebyshev polynomials, smoother and subspace filters in FP64 (oracle; test
infrastructure only).

Paper: arXiv:2103.05034.
  Sec. 3.2, Eq. (23): T_n(x) = cos(n arccos x), produced by the recurrence
           T_0 = 1, T_1 = x, T_{n+1} = 2 x T_n - T_{n-1}; the interval [a,b]
           maps to [-1,1] by x = 2(y-a)/(b-a) - 1.
  Sec. 3.2, Eq. (24): S_cheb([a,b],N) = [c_0/2 + sum_j c_j T_j(x(M^dag M))] M^dag
  Sec. 3.2, Eq. (25): c_j = (2/N) sum_{k=0}^{N-1} f(y(cos theta_k)) cos(j theta_k),
           theta_k = pi (k + 1/2) / N, f(y) = 1/y
  Sec. 3.4, Eq. (34): pre-filter T_m(2(M^dag M - lambda_lo)/(lambda_max - lambda_lo) - 1) eta
  Sec. 3.4, Eqs. (35), (37): phi_k = T_{k Delta}(2 M^dag M / lambda_max - 1) phi_0

Readings:
  * Eq. (24) sums j = 1..N, but c_N vanishes identically because
    cos(N theta_k) = cos(pi (k + 1/2)) = 0; the sum here stops at N-1, which is
    the same polynomial and saves one application of M^dag M.
  * y(x) = a + (b - a)(x + 1)/2 is the inverse of the interval map.
  * Eq. (34) prints the denominator as lambda_{max - lambda_lo}; it is read as
    (lambda_max - lambda_lo).  Eq. (37) repeats the pre-filter with lambda_max
    alone; Eq. (34)'s form is used.
  * Each filtered vector is returned normalised to unit norm (the paper does
    not say; the deflation space only depends on directions).
"""
from __future__ import annotations

import numpy as np

from . import dwf


def cheb_T(n, x):
    """T_n(x) for scalars/arrays by the three-term recurrence."""
    x = np.asarray(x, dtype=float)
    if n == 0:
        return np.ones_like(x)
    t0, t1 = np.ones_like(x), x.copy()
    for _ in range(n - 1):
        t0, t1 = t1, 2 * x * t1 - t0
    return t1


def smoother_coeffs(a, b, N):
    """c_0..c_N of Eq. (25) for f(y) = 1/y on [a, b]."""
    k = np.arange(N)
    theta = np.pi * (k + 0.5) / N
    y = a + (b - a) * (np.cos(theta) + 1) / 2
    f = 1.0 / y
    return np.array([(2.0 / N) * np.sum(f * np.cos(j * theta)) for j in range(N + 1)])


def smoother_scalar(lam, a, b, N):
    """The scalar polynomial p(lam) = c_0/2 + sum_{j=1}^{N-1} c_j T_j(x(lam)) of Eq. (24)."""
    c = smoother_coeffs(a, b, N)
    x = 2 * (np.asarray(lam, float) - a) / (b - a) - 1
    return 0.5 * c[0] + sum(c[j] * cheb_T(j, x) for j in range(1, N))


def poly_apply(apply_A, v, coeffs, lo, hi):
    """sum_j coeffs[j] T_j(x(A)) v, x(A) = 2(A - lo)/(hi - lo) - 1, with the
    T_j v generated by the recurrence.  Returns (result, applications of A)."""
    n = len(coeffs)
    xA = lambda w: (2.0 / (hi - lo)) * apply_A(w) - ((hi + lo) / (hi - lo)) * w
    t_prev = v
    out = coeffs[0] * v
    nA = 0
    if n > 1:
        t_cur = xA(v)
        nA += 1
        out = out + coeffs[1] * t_cur
        for j in range(2, n):
            t_next = 2 * xA(t_cur) - t_prev
            nA += 1
            t_prev, t_cur = t_cur, t_next
            out = out + coeffs[j] * t_cur
    return out, nA


def smoother_apply(apply_M, apply_Mdag, r, a, b, N):
    """S_cheb([a,b],N) r of Eq. (24): [c_0/2 + sum_{j<N} c_j T_j(x(M^dag M))] M^dag r.
    Returns (z, applications of M or M^dag)."""
    c = smoother_coeffs(a, b, N)
    coeffs = np.concatenate([[0.5 * c[0]], c[1:N]])
    v = apply_Mdag(r)
    z, nA = poly_apply(lambda w: apply_Mdag(apply_M(w)), v, coeffs, a, b)
    return z, 1 + 2 * nA


def cheby_filter(apply_A, v, order, lo, hi):
    """T_order(x(A)) v with x(A) = 2(A - lo)/(hi - lo) - 1, by the recurrence."""
    coeffs = np.zeros(order + 1)
    coeffs[order] = 1.0
    out, _ = poly_apply(apply_A, v, coeffs, lo, hi)
    return out


def recursive_basis(apply_A, eta, m, delta, nvec, lam_lo, lam_max):
    """The filtered vectors of Sec. 3.4: phi_0 from the order-m pre-filter on
    [lam_lo, lam_max] (Eq. 34), then phi_k = T_{k delta}(2A/lam_max - 1) phi_0
    for k = 1..nvec-1 (Eqs. 35, 37), taken as snapshots of one recurrence.
    Returns a list of unit-norm vectors."""
    phi0 = cheby_filter(apply_A, eta, m, lam_lo, lam_max)
    phi0 = phi0 / np.sqrt(dwf.norm2(phi0))
    out = [phi0.copy()]
    xA = lambda w: (2.0 / lam_max) * apply_A(w) - w
    t_prev, t_cur = phi0, xA(phi0)
    n = 1
    for k in range(1, nvec):
        while n < k * delta:
            t_prev, t_cur = t_cur, 2 * xA(t_cur) - t_prev
            n += 1
        out.append(t_cur / np.sqrt(dwf.norm2(t_cur)))
    return out
