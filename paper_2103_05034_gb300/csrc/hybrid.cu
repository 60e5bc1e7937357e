// Hybrid three-level multigrid (arXiv:2103.05034, Sec. 4, Algorithm F,
// Hybrid-M^dag M): a 4D coarsening of the Wilson operator D_W (Eq. 1) that
// keeps the fifth dimension, giving a coarse domain wall operator M_1 on the
// level-1 lattice; a second coarsening of H_1 = Gamma5_1 M_1 on blocks of one
// level-1 site spanning all s (the level-2 stencil, solved like the HDCR
// coarse operator); a fixed-iteration W-cycle (two coarse-coarse corrections
// per coarse grid step).
//
// Layouts.  4D basis: nb4 4D fields stored as the s-slices of one full field
// with Ls = nb4 ([parity][Vh][12][nb4], vector innermost), so that the
// hopping kernels of a context with Ls = nb4 apply D_hop to all of them at
// once (D_hop acts on every s-slice alike).  Level-1 vectors: FP32
// [nc1][nb4][Ls][nvec].  Level-2 basis: FP32 [nc1][nb4][Ls][nb2] (a level-1
// multi-vector).  Level-2 vectors: FP32 [nc1][nb2].
#include <math.h>
#include <string.h>

#include <chrono>
#include <new>
#include <vector>

#include "coarse_internal.cuh"

struct dwf_hybrid {
  dwf_ctx* ctx;            // fine context
  dwf_mg_params p;         // fine-level and level-2 solver parameters
  dwf_hybrid_params hp;
  BlockGeom g;             // 4D blocks on the fine field (Ls = fine Ls)
  BlockGeom g4;            // the same blocks on the 4D basis (Ls = nb4)
  int nb4, np4, nb2, np2, Ls;
  int64_t nc1;             // level-1 sites
  double2* phi64;          // 4D basis, FP64
  float2* phi32;           // 4D basis, FP32
  dwf_coarse* C1;          // B on the level-1 lattice (nb = nb4)
  float2* Phi2;            // level-2 basis
  dwf_coarse* C2;          // level-2 stencil (nb = nb2)
  void* w[10];
  size_t wb[10];
  double setup_seconds, coarse_op_seconds;
};

namespace hyb {

using dwfmg::BlockGeom;
using dwfmg::block_site_offset;

// (1 + gamma_5)/2 on the first nplus slices, (1 - gamma_5)/2 on the rest, in
// place: gamma_5 = diag(1, 1, -1, -1), so the projection keeps spins 0, 1 or
// 2, 3 (colour-spin index c = 3 spin + colour, c < 6 for spins 0, 1).
template <class T>
__global__ void k_chiral4(T* X, long long n, int nv, int nplus) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int v = (int)(e % nv);
  const int c = (int)((e / nv) % 12);
  const bool keep = v < nplus ? c < 6 : c >= 6;
  if (!keep) {
    T z;
    z.x = 0;
    z.y = 0;
    X[e] = z;
  }
}

// Term d of -1/2 D_hop on 4D blocks for nv 4D fields stored as slices: d =
// 1+2mu (2+2mu) the hop from x+mu (x-mu) at sites on the +mu (-mu) face of
// their block, d = 0 the sum of the hops whose neighbour lies in the block.
// One thread per (parity, site, slice); FP64.
__global__ void __launch_bounds__(128) k_hop4_part(double2* out, const double2* in, const double2* links0,
                                                   const double2* links1, BlockGeom g, int nv, int d) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2LL * g.Vh * nv) return;
  const int v = (int)(e % nv);
  const long long ps = e / nv;
  const int p = (int)(ps / g.Vh);
  const int h = (int)(ps - (long long)p * g.Vh);
  int rem = h / g.Lxh;
  const int xh = h - rem * g.Lxh;
  int x[4];
  x[1] = rem % g.L[1];
  rem /= g.L[1];
  x[2] = rem % g.L[2];
  x[3] = rem / g.L[2];
  x[0] = 2 * xh + ((x[1] + x[2] + x[3] + p) & 1);
  cpx<double> acc[12], ps12[12];
#pragma unroll
  for (int c = 0; c < 12; c++) acc[c] = cmake<double>(0, 0);
  for (int dir = 1; dir <= 8; dir++) {
    const int mu = (dir - 1) >> 1;
    const bool fwd = ((dir - 1) & 1) == 0;
    const bool face = fwd ? (x[mu] % g.b[mu] == g.b[mu] - 1) : (x[mu] % g.b[mu] == 0);
    if (d == 0 ? face : (dir != d || !face)) continue;
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] = fwd ? (y[mu] + 1 == g.L[mu] ? 0 : y[mu] + 1) : (y[mu] == 0 ? g.L[mu] - 1 : y[mu] - 1);
    const long long ylex = y[0] + (long long)g.L[0] * (y[1] + (long long)g.L[1] * (y[2] + (long long)g.L[2] * y[3]));
    const double2* src = in + ((long long)(1 - p) * g.Vh + (ylex >> 1)) * 12 * nv + v;
#pragma unroll
    for (int c = 0; c < 12; c++) ps12[c] = ld_c(src + (long long)c * nv);
    cpx<double> U[9];
    const double2* lk = (p ? links1 : links0) + ((long long)h * 8 + 2 * mu + (fwd ? 0 : 1)) * 9;
#pragma unroll
    for (int a = 0; a < 9; a++) U[a] = ld_c(lk + a);
    const double sg = fwd ? 1.0 : -1.0;
    switch (mu) {
      case 0:
        dwfk::hop_dir<double, 0>(acc, ps12, U, sg);
        break;
      case 1:
        dwfk::hop_dir<double, 1>(acc, ps12, U, sg);
        break;
      case 2:
        dwfk::hop_dir<double, 2>(acc, ps12, U, sg);
        break;
      default:
        dwfk::hop_dir<double, 3>(acc, ps12, U, sg);
        break;
    }
  }
  double2* o = out + ps * 12 * nv + v;
#pragma unroll
  for (int c = 0; c < 12; c++) st_c(o + (long long)c * nv, cmake<double>(-0.5 * acc[c].re, -0.5 * acc[c].im));
}

// G[xc][j][k] = sum over the block's sites and colour-spin of conj(X_j) Y_k
// for nv slices of FP64 4D fields.  One CTA per block.
constexpr int G4_MAXNV = 24;
__global__ void __launch_bounds__(256) k_gram4(double2* G, long long gstride, const double2* X, const double2* Y,
                                               BlockGeom g, int nv) {
  __shared__ cpx<double> sx[12 * G4_MAXNV], sy[12 * G4_MAXNV];
  const int xc = blockIdx.x;
  const int nent = nv * nv;
  cpx<double> acc[3];
  for (int q = 0; q < 3; q++) acc[q] = cmake<double>(0, 0);
  for (int i = 0; i < g.b4; i++) {
    bool face;
    const long long off = block_site_offset(g, xc, i, 0, &face);
    for (int t = threadIdx.x; t < 12 * nv; t += blockDim.x) {
      sx[t] = ld_c(X + off + t);
      sy[t] = ld_c(Y + off + t);
    }
    __syncthreads();
    for (int q = 0; q < 3; q++) {
      const int ent = threadIdx.x + q * blockDim.x;
      if (ent >= nent) break;
      const int j = ent / nv, k = ent - j * nv;
      double re = acc[q].re, im = acc[q].im;
      for (int c = 0; c < 12; c++) {
        const cpx<double> a = sx[c * nv + j], b = sy[c * nv + k];
        re = fma(a.re, b.re, re);
        re = fma(a.im, b.im, re);
        im = fma(a.re, b.im, im);
        im = fma(-a.im, b.re, im);
      }
      acc[q] = cmake(re, im);
    }
    __syncthreads();
  }
  for (int q = 0; q < 3; q++) {
    const int ent = threadIdx.x + q * blockDim.x;
    if (ent < nent) G[(long long)xc * gstride + ent] = make_double2(acc[q].re, acc[q].im);
  }
}

// x_k <- sum_{j <= k} x_j Rinv[xc][j][k] on every (site, colour-spin) row of
// the block (FP64 4D basis in place; Rinv upper triangular and zero across
// chirality groups).
__global__ void __launch_bounds__(256) k_update4(double2* X, const double2* Rinv, BlockGeom g, int nv) {
  __shared__ double2 R[G4_MAXNV * G4_MAXNV];
  const int xc = blockIdx.x;
  for (int t = threadIdx.x; t < nv * nv; t += blockDim.x) R[t] = Rinv[(long long)xc * nv * nv + t];
  __syncthreads();
  for (int row = threadIdx.x; row < g.b4 * 12; row += blockDim.x) {
    const int i = row / 12, c = row - i * 12;
    bool face;
    double2* x = X + block_site_offset(g, xc, i, 0, &face) + (long long)c * nv;
    double2 v[G4_MAXNV];
    for (int j = 0; j < nv; j++) v[j] = x[j];
    for (int k = 0; k < nv; k++) {
      double re = 0, im = 0;
      for (int j = 0; j <= k; j++) {
        const double2 m = R[j * nv + k];
        re += v[j].x * m.x - v[j].y * m.y;
        im += v[j].x * m.y + v[j].y * m.x;
      }
      x[k] = make_double2(re, im);
    }
  }
}

// Level-1 restriction P1^dag: out[xc][k][s][vec] = sum over the block's sites
// and colour-spin of conj(phi_k) psi_vec(s).  One CTA per (block, vector),
// one thread per (k, s); FP32.
__global__ void k_restrict4(float2* out, const float2* psi, long long fstride, const float2* phi, BlockGeom g,
                            BlockGeom g4, int nvec) {
  extern __shared__ cpx<float> sm4[];
  const int nb4 = g4.Ls, Ls = g.Ls;
  cpx<float>* sphi = sm4;
  cpx<float>* spsi = sm4 + 12 * nb4;
  const int xc = blockIdx.x, vec = blockIdx.y;
  const int t = threadIdx.x;
  const int k = t / Ls, s = t - k * Ls;
  float re = 0.f, im = 0.f;
  const float2* pv = psi + (long long)vec * fstride;
  for (int i = 0; i < g.b4; i++) {
    bool face;
    const long long offp = block_site_offset(g, xc, i, 0, &face);
    const long long off4 = block_site_offset(g4, xc, i, 0, &face);
    for (int q = t; q < 12 * nb4; q += blockDim.x) sphi[q] = ld_c(phi + off4 + q);
    for (int q = t; q < 12 * Ls; q += blockDim.x) spsi[q] = ld_c(pv + offp + q);
    __syncthreads();
    if (k < nb4) {
#pragma unroll 4
      for (int c = 0; c < 12; c++) {
        const cpx<float> a = sphi[c * nb4 + k], b = spsi[c * Ls + s];
        re = fmaf(a.re, b.re, re);
        re = fmaf(a.im, b.im, re);
        im = fmaf(a.re, b.im, im);
        im = fmaf(-a.im, b.re, im);
      }
    }
    __syncthreads();
  }
  if (k < nb4) out[(((long long)xc * nb4 + k) * Ls + s) * nvec + vec] = make_float2(re, im);
}

// Level-1 prolongation P1: psi_vec(x, c, s) (+)= sum_k phi_k(x, c) v(xc, k, s, vec).
__global__ void k_prolong4(float2* psi, long long fstride, const float2* v, const float2* phi, BlockGeom g,
                           BlockGeom g4, int nvec, int accumulate) {
  extern __shared__ cpx<float> sm4[];
  const int nb4 = g4.Ls, Ls = g.Ls;
  cpx<float>* sv = sm4;
  cpx<float>* sphi = sm4 + nb4 * Ls;
  const int xc = blockIdx.x, vec = blockIdx.y;
  const int t = threadIdx.x;
  for (int q = t; q < nb4 * Ls; q += blockDim.x) sv[q] = ld_c(v + ((long long)xc * nb4 * Ls + q) * nvec + vec);
  float2* pv = psi + (long long)vec * fstride;
  for (int i = 0; i < g.b4; i++) {
    bool face;
    const long long offp = block_site_offset(g, xc, i, 0, &face);
    const long long off4 = block_site_offset(g4, xc, i, 0, &face);
    __syncthreads();
    for (int q = t; q < 12 * nb4; q += blockDim.x) sphi[q] = ld_c(phi + off4 + q);
    __syncthreads();
    for (int q = t; q < 12 * Ls; q += blockDim.x) {
      const int c = q / Ls, s = q - c * Ls;
      float re = 0.f, im = 0.f;
      for (int k = 0; k < nb4; k++) {
        const cpx<float> a = sphi[c * nb4 + k], b = sv[k * Ls + s];
        re = fmaf(a.re, b.re, re);
        re = fmaf(-a.im, b.im, re);
        im = fmaf(a.re, b.im, im);
        im = fmaf(a.im, b.re, im);
      }
      if (accumulate) {
        const float2 o = pv[offp + q];
        re += o.x;
        im += o.y;
      }
      pv[offp + q] = make_float2(re, im);
    }
  }
}

// Fifth-dimension part of M_1 added to a hopping result, with Gamma5_1 on the
// output when herm: val(s) = hop(s) + (5 - M5) in(s) + [chi = +1: -in(s-1),
// or mf in(Ls-1) at s = 0; chi = -1: -in(s+1), or mf in(0) at s = Ls-1]
// (Eq. 4 on one chirality), out(s) = chi val(Ls-1-s) for H_1.  out may equal
// hop when herm = 0 (each thread reads only its own hop element).
template <class TO, class TH>
__global__ void k_l1_tail(TO* out, const TH* hop, const float2* in, long long n, int nb4, int np4, int Ls, int nvec,
                          double d5, double mf, int herm) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int v = (int)(e % nvec);
  const long long t = e / nvec;
  const int s = (int)(t % Ls);
  const long long xk = t / Ls;
  const int k = (int)(xk % nb4);
  const bool plus = k < np4;
  const int ss = herm ? Ls - 1 - s : s;
  const long long base = xk * Ls * nvec + v;
  const TH hv = hop[base + (long long)ss * nvec];
  const cpx<double> h = cmake<double>(hv.x, hv.y);
  const float2 a = in[base + (long long)ss * nvec];
  int sn;
  double co;
  if (plus) {
    sn = ss >= 1 ? ss - 1 : Ls - 1;
    co = ss >= 1 ? -1.0 : mf;
  } else {
    sn = ss <= Ls - 2 ? ss + 1 : 0;
    co = ss <= Ls - 2 ? -1.0 : mf;
  }
  const float2 b = in[base + (long long)sn * nvec];
  double re = h.re + d5 * a.x + co * b.x;
  double im = h.im + d5 * a.y + co * b.y;
  if (herm && !plus) {
    re = -re;
    im = -im;
  }
  TO o;
  o.x = re;
  o.y = im;
  out[e] = o;
}

// (1 + sigma Gamma5_1)/2 in place on a level-1 multi-vector, sigma = +1 for
// the first np2 vectors and -1 for the rest; one thread per (s, Ls-1-s) pair.
__global__ void k_l1_chiral(float2* X, long long nxk, int nb4, int np4, int Ls, int nvec, int np2) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int half = Ls / 2;
  if (e >= nxk * half * nvec) return;
  const int v = (int)(e % nvec);
  const long long t = e / nvec;
  const int s = (int)(t % half);
  const long long xk = t / half;
  const int k = (int)(xk % nb4);
  const float sc = ((k < np4) == (v < np2)) ? 1.f : -1.f;
  float2* a = X + (xk * Ls + s) * nvec + v;
  float2* b = X + (xk * Ls + (Ls - 1 - s)) * nvec + v;
  const float2 va = *a, vb = *b;
  *a = make_float2(0.5f * (va.x + sc * vb.x), 0.5f * (va.y + sc * vb.y));
  *b = make_float2(0.5f * (vb.x + sc * va.x), 0.5f * (vb.y + sc * va.y));
}

// G[x*gstride + goff + i*nb + j] = sum_q conj(X[x][q][i]) Y'[x][q][j] over the
// nq = nb4 Ls rows q = (k, s) of one level-1 site, Y' = Gamma5_1 Y when g5
// (row (k, s) takes chi_k Y[(k, Ls-1-s)]).  One CTA per site, rows staged in
// chunks of 16; FP64 sums.
constexpr int GS_ROWS = 16;
template <class TY>
__global__ void __launch_bounds__(256) k_gram_site(double2* G, long long gstride, long long goff, const float2* X,
                                                   const TY* Y, int nq, int nb, int g5, int np4, int Ls) {
  __shared__ cpx<double> sx[GS_ROWS][64], sy[GS_ROWS][64];
  const long long x = blockIdx.x;
  const int nent = nb * nb;
  cpx<double> acc[16];
#pragma unroll
  for (int q = 0; q < 16; q++) acc[q] = cmake<double>(0, 0);
  for (int q0 = 0; q0 < nq; q0 += GS_ROWS) {
    const int nr = min(GS_ROWS, nq - q0);
    for (int t = threadIdx.x; t < nr * nb; t += blockDim.x) {
      const int r = t / nb, i = t - r * nb;
      const int q = q0 + r;
      const float2 a = X[((long long)x * nq + q) * nb + i];
      sx[r][i] = cmake<double>(a.x, a.y);
      int qy = q;
      double sg = 1.0;
      if (g5) {
        const int k = q / Ls, s = q - k * Ls;
        qy = k * Ls + (Ls - 1 - s);
        sg = k < np4 ? 1.0 : -1.0;
      }
      const TY b = Y[((long long)x * nq + qy) * nb + i];
      sy[r][i] = cmake<double>(sg * (double)b.x, sg * (double)b.y);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 16; u++) {
      const int ent = threadIdx.x + u * blockDim.x;
      if (ent < nent) {
        const int i = ent / nb, j = ent - i * nb;
        double re = acc[u].re, im = acc[u].im;
        for (int r = 0; r < nr; r++) {
          const cpx<double> a = sx[r][i], b = sy[r][j];
          re = fma(a.re, b.re, re);
          re = fma(a.im, b.im, re);
          im = fma(a.re, b.im, im);
          im = fma(-a.im, b.re, im);
        }
        acc[u] = cmake(re, im);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 16; u++) {
    const int ent = threadIdx.x + u * blockDim.x;
    if (ent < nent) G[x * gstride + goff + ent] = make_double2(acc[u].re, acc[u].im);
  }
}

// X[x][q][k] <- sum_{j <= k} X[x][q][j] Rinv[x][j][k] on every row q of the
// site (level-2 basis in place, FP64 arithmetic); rows staged in chunks.
__global__ void __launch_bounds__(256) k_update_site(float2* X, const double2* Rinv, int nq, int nb) {
  __shared__ float2 sr[GS_ROWS][64];
  const long long x = blockIdx.x;
  const double2* R = Rinv + x * nb * nb;
  for (int q0 = 0; q0 < nq; q0 += GS_ROWS) {
    const int nr = min(GS_ROWS, nq - q0);
    for (int t = threadIdx.x; t < nr * nb; t += blockDim.x) {
      const int r = t / nb, i = t - r * nb;
      sr[r][i] = X[((long long)x * nq + q0 + r) * nb + i];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nr * nb; t += blockDim.x) {
      const int r = t / nb, k = t - r * nb;
      double re = 0, im = 0;
      for (int j = 0; j <= k; j++) {
        const double2 m = __ldg(R + j * nb + k);
        const float2 v = sr[r][j];
        re += (double)v.x * m.x - (double)v.y * m.y;
        im += (double)v.x * m.y + (double)v.y * m.x;
      }
      X[((long long)x * nq + q0 + r) * nb + k] = make_float2((float)re, (float)im);
    }
    __syncthreads();
  }
}

// Level-2 restriction P2^dag: out[x][i] = sum_q conj(Phi[x][q][i]) v[x][q].
__global__ void k_restrict2(float2* out, const float2* v, const float2* Phi, long long nc, int nq, int nb) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nc * nb) return;
  const long long x = e / nb;
  const int i = (int)(e - x * nb);
  float re = 0.f, im = 0.f;
  const float2* ph = Phi + x * nq * nb + i;
  const float2* vv = v + x * nq;
  for (int q = 0; q < nq; q++) {
    const float2 a = ph[(long long)q * nb], b = vv[q];
    re = fmaf(a.x, b.x, re);
    re = fmaf(a.y, b.y, re);
    im = fmaf(a.x, b.y, im);
    im = fmaf(-a.y, b.x, im);
  }
  out[e] = make_float2(re, im);
}

// Level-2 prolongation P2: v[x][q] (+)= sum_i Phi[x][q][i] e[x][i].
__global__ void k_prolong2(float2* v, const float2* e2, const float2* Phi, long long nc, int nq, int nb,
                           int accumulate) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nc * nq) return;
  const long long x = e / nq;
  const float2* ph = Phi + e * nb;
  const float2* ee = e2 + x * nb;
  float re = 0.f, im = 0.f;
  for (int i = 0; i < nb; i++) {
    const float2 a = ph[i], b = ee[i];
    re = fmaf(a.x, b.x, re);
    re = fmaf(-a.y, b.y, re);
    im = fmaf(a.x, b.y, im);
    im = fmaf(a.y, b.x, im);
  }
  if (accumulate) {
    const float2 o = v[e];
    re += o.x;
    im += o.y;
  }
  v[e] = make_float2(re, im);
}

// One direction of the level-1 hop: out[x][j][r] = sum_k B[x][d][j][k] in[x+d][k][r]
// (FP64 stencil and sums, FP32 input).
__global__ void k_dir_apply(double2* out, const float2* in, const double2* B, int Lc0, int Lc1, int Lc2, int Lc3,
                            int nb, int nrhs, int d) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nc = (long long)Lc0 * Lc1 * Lc2 * Lc3;
  if (e >= nc * nb * nrhs) return;
  const int r = (int)(e % nrhs);
  const long long t = e / nrhs;
  const int j = (int)(t % nb);
  const int x = (int)(t / nb);
  const int Lc[4] = {Lc0, Lc1, Lc2, Lc3};
  const int y = dwfmg::coarse_nbr(Lc, x, d);
  const double2* Bd = B + (((long long)x * 9 + d) * nb + j) * nb;
  const float2* v = in + (long long)y * nb * nrhs + r;
  double re = 0, im = 0;
  for (int k = 0; k < nb; k++) {
    const double2 a = __ldg(Bd + k);
    const float2 b = v[(long long)k * nrhs];
    re = fma(a.x, (double)b.x, re);
    re = fma(-a.y, (double)b.y, re);
    im = fma(a.x, (double)b.y, im);
    im = fma(a.y, (double)b.x, im);
  }
  out[e] = make_double2(re, im);
}

// out[i] = in[i * stride]: the first vector of a multi-vector.
__global__ void k_column(double2* out, const double2* in, long long n, int stride) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = in[e * stride];
}

}  // namespace hyb

namespace {

using dwfmg::BlockGeom;

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double sec() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Hybrid workspaces: setup temporaries (freed after the setup) and the
// level-1 arena of the solve.
enum { HW_F0, HW_F1, HW_F2, HW_F3, HW_F4, HW_G, HW_R, HW_FAIL, HW_ARENA, HW_L2 };

void* hws(dwf_hybrid* H, int slot, size_t bytes) {
  if (H->wb[slot] < bytes || !H->w[slot]) {
    if (H->w[slot]) cudaFree(H->w[slot]);
    H->w[slot] = nullptr;
    H->wb[slot] = 0;
    if (cudaMalloc(&H->w[slot], bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    H->wb[slot] = bytes;
  }
  return H->w[slot];
}

void hws_free(dwf_hybrid* H, int slot) {
  if (H->w[slot]) cudaFree(H->w[slot]);
  H->w[slot] = nullptr;
  H->wb[slot] = 0;
}

int64_t n1(const dwf_hybrid* H) { return H->nc1 * H->nb4 * H->Ls; }       // one level-1 vector
int64_t fine_elems(const dwf_ctx* c) { return 2 * c->g.Vh * 12 * c->g.Ls; }

// One application of D_W(m)/(4+m) = 1 - kappa D_hop (kappa = 1/(2(4+m)),
// Eq. 1) or of its adjoint to the nb4 4D fields held as the slices of a full
// field of the Ls = nb4 context; with cf the result feeds cf's Chebyshev step
// in the second (odd-parity) launch and in the first, both parities being
// outputs of this application.
int wilson_hat(dwf_ctx* c4, void* out, const void* in, double kappa, int dagger, cudaStream_t st,
               const ChebFuse* cf) {
  const int64_t he = c4->g.Vh * 12 * c4->g.Ls;
  const size_t cb = sizeof(float2);
  for (int po = 0; po < 2; po++) {
    HopLaunch h;
    memset(&h, 0, sizeof(h));
    h.out = cf ? nullptr : (char*)out + po * he * cb;
    h.in = (const char*)in + (1 - po) * he * cb;
    h.aux = (const char*)in + po * he * cb;
    h.out_parity = po;
    h.dagger = dagger;
    h.nrhs = 1;
    h.rhs_stride = 2 * he;
    h.alpha = -kappa;
    h.aux_mode = 1;
    if (cf) {
      h.cheb_x = (const char*)cf->x + po * he * cb;
      h.cheb_tp = (char*)cf->tp + po * he * cb;
      h.cheb_acc = cf->acc ? (char*)cf->acc + po * he * cb : nullptr;
      h.cheb_ta = cf->ta;
      h.cheb_tb = cf->tb;
      h.cheb_cacc = cf->cacc;
    }
    int rc = launch_hop(c4, h, DWF_F32, st, nullptr);
    if (rc) return rc;
  }
  return DWF_OK;
}

// Rescale a Chebyshev pair (T_{k-1}, T_k) by a common factor when T_k has
// grown past 1e15 (the recurrence is linear, so directions are kept).
int rescale_pair(dwf_ctx* c, void* tp, void* tc, int64_t n, cudaStream_t st) {
  int rc = norm2_dev(c, tc, n, DWF_F32, S_TMP3, st);
  if (rc) return rc;
  rc = read_scalars(c, S_TMP3, 1, st);
  if (rc) return rc;
  const double nn = c->hscal[S_TMP3];
  if (!isfinite(nn)) return dwf_fail(c, DWF_ERANGE, "Chebyshev filter overflow: spectrum outside [lo, hi]");
  if (nn > 1e30) {
    const double f = 1.0 / sqrt(nn);
    rc = blas_axpby(c, 0.0, tc, DWF_F32, f, tc, DWF_F32, n, st);
    if (rc == DWF_OK) rc = blas_axpby(c, 0.0, tp, DWF_F32, f, tp, DWF_F32, n, st);
  }
  return rc;
}

// Block Cholesky-QR of the FP64 4D basis in place (three passes, the first
// shifted by 1e-6 of the largest Gram diagonal: the vectors come from an FP32
// filter and can be dependent to that precision on a block).
int ortho4(dwf_hybrid* H, cudaStream_t st) {
  dwf_ctx* c = H->ctx;
  const int nv = H->nb4;
  const size_t gb = (size_t)H->nc1 * nv * nv * sizeof(double2);
  double2* G = (double2*)hws(H, HW_G, gb);
  double2* R = (double2*)hws(H, HW_R, gb);
  int* fail = (int*)hws(H, HW_FAIL, 4 * sizeof(int));
  if (!G || !R || !fail) return dwf_fail(c, DWF_ENOMEM, "hybrid orthonormalisation workspace");
  for (int pass = 0; pass < 3; pass++) {
    c->launches += 3;
    hyb::k_gram4<<<(unsigned)H->nc1, 256, 0, st>>>(G, (long long)nv * nv, H->phi64, H->phi64, H->g4, nv);
    DWF_CUDA(c, cudaMemsetAsync(R, 0, gb, st));
    DWF_CUDA(c, cudaMemsetAsync(fail, 0, sizeof(int), st));
    dwfmg::k_block_cholinv<<<dim3((unsigned)H->nc1, 2), 32, 0, st>>>(G, R, nv, H->np4, fail, pass == 0 ? 1e-6 : 0.0);
    hyb::k_update4<<<(unsigned)H->nc1, 256, 0, st>>>(H->phi64, R, H->g4, nv);
    int hf = 0;
    DWF_CUDA(c, cudaMemcpyAsync(&hf, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CUDA(c, cudaStreamSynchronize(st));
    if (hf) return dwf_fail(c, DWF_ERANGE, "4D basis vectors linearly dependent on a block");
  }
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

// Per-site Cholesky-QR of the level-2 basis in place (FP64 Gram matrices and
// updates on FP32 storage; three passes, the first shifted).
int ortho2(dwf_hybrid* H, cudaStream_t st) {
  dwf_ctx* c = H->ctx;
  const int nb = H->nb2, nq = H->nb4 * H->Ls;
  const size_t gb = (size_t)H->nc1 * nb * nb * sizeof(double2);
  double2* G = (double2*)hws(H, HW_G, gb);
  double2* R = (double2*)hws(H, HW_R, gb);
  int* fail = (int*)hws(H, HW_FAIL, 4 * sizeof(int));
  if (!G || !R || !fail) return dwf_fail(c, DWF_ENOMEM, "hybrid orthonormalisation workspace");
  for (int pass = 0; pass < 3; pass++) {
    c->launches += 3;
    hyb::k_gram_site<float2><<<(unsigned)H->nc1, 256, 0, st>>>(G, (long long)nb * nb, 0, H->Phi2, H->Phi2, nq, nb,
                                                                0, H->np4, H->Ls);
    DWF_CUDA(c, cudaMemsetAsync(R, 0, gb, st));
    DWF_CUDA(c, cudaMemsetAsync(fail, 0, sizeof(int), st));
    dwfmg::k_block_cholinv<<<dim3((unsigned)H->nc1, 2), 32, 0, st>>>(G, R, nb, H->np2, fail, pass == 0 ? 1e-5 : 0.0);
    hyb::k_update_site<<<(unsigned)H->nc1, 256, 0, st>>>(H->Phi2, R, nq, nb);
    int hf = 0;
    DWF_CUDA(c, cudaMemcpyAsync(&hf, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CUDA(c, cudaStreamSynchronize(st));
    if (hf) return dwf_fail(c, DWF_ERANGE, "level-2 basis vectors linearly dependent on a site");
  }
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

}  // namespace

// ---------------------------------------------------------------------- level operators
// M_1 (herm = 0) or H_1 (herm = 1) on nvec level-1 vectors; tmp holds the hop.
int hybrid_l1_apply(dwf_hybrid* H, float2* out, const float2* in, int nvec, int herm, float2* tmp, cudaStream_t st) {
  int rc = coarse_apply_dev(H->C1, tmp, in, H->Ls * nvec, st);
  if (rc) return rc;
  const long long n = (long long)n1(H) * nvec;
  H->ctx->launches++;
  hyb::k_l1_tail<float2, float2><<<nblk(n), 256, 0, st>>>(out, tmp, in, n, H->nb4, H->np4, H->Ls, nvec,
                                                          5.0 - H->ctx->M5, H->p.mf, herm);
  return DWF_OK;
}

int hybrid_restrict1(dwf_hybrid* H, float2* out, const float2* psi, int nvec, cudaStream_t st) {
  const int nt = ((H->nb4 * H->Ls + 31) / 32) * 32;
  const size_t sm = (size_t)12 * (H->nb4 + H->Ls) * sizeof(cpx<float>);
  H->ctx->launches++;
  hyb::k_restrict4<<<dim3((unsigned)H->nc1, nvec), nt, sm, st>>>(out, psi, fine_elems(H->ctx), H->phi32, H->g,
                                                                 H->g4, nvec);
  return DWF_OK;
}

int hybrid_prolong1(dwf_hybrid* H, float2* psi, const float2* v, int nvec, int accumulate, cudaStream_t st) {
  const size_t sm = (size_t)(H->nb4 * H->Ls + 12 * H->nb4) * sizeof(cpx<float>);
  H->ctx->launches++;
  hyb::k_prolong4<<<dim3((unsigned)H->nc1, nvec), 256, sm, st>>>(psi, fine_elems(H->ctx), v, H->phi32, H->g, H->g4,
                                                                 nvec, accumulate);
  return DWF_OK;
}

int hybrid_restrict2(dwf_hybrid* H, float2* out, const float2* v, cudaStream_t st) {
  H->ctx->launches++;
  hyb::k_restrict2<<<nblk(H->nc1 * H->nb2), 256, 0, st>>>(out, v, H->Phi2, H->nc1, H->nb4 * H->Ls, H->nb2);
  return DWF_OK;
}

int hybrid_prolong2(dwf_hybrid* H, float2* v, const float2* e2, int accumulate, cudaStream_t st) {
  H->ctx->launches++;
  hyb::k_prolong2<<<nblk(n1(H)), 256, 0, st>>>(v, e2, H->Phi2, H->nc1, H->nb4 * H->Ls, H->nb2, accumulate);
  return DWF_OK;
}

namespace {

// Level-1 arena: single level-1 vectors for the solve (see the slot names).
enum { A_R1, A_E1, A_RES, A_HOP, A_X, A_RR, A_S2, A_V, A_TP, A_TC, A_AX, A_TMP, A_ZW };

float2* arena(dwf_hybrid* H, int slot) {
  return (float2*)H->w[HW_ARENA] + (size_t)slot * n1(H);
}

int arena_ready(dwf_hybrid* H) {
  const size_t nslots = A_ZW + 2 * (size_t)H->hp.kcycle;
  if (!hws(H, HW_ARENA, nslots * n1(H) * sizeof(float2)) ||
      !hws(H, HW_L2, 2 * (size_t)H->nc1 * H->nb2 * sizeof(float2)))
    return dwf_fail(H->ctx, DWF_ENOMEM, "hybrid level-1 workspace");
  return DWF_OK;
}

// Chebyshev smoother of Eqs. (24)-(25) with M = M^dag = H_1 on one level-1
// vector: z = [c0/2 + sum_{j=1}^{N-1} c_j T_j(y(H_1^2))] H_1 r.
int l1_smoother(dwf_hybrid* H, float2* z, const float2* r, cudaStream_t st) {
  dwf_ctx* c = H->ctx;
  const double a = H->hp.smooth1_lo, b = H->hp.smooth1_hi;
  const int N = H->hp.smooth1_order;
  const int64_t n = n1(H);
  std::vector<double> cf(N + 1);
  for (int j = 0; j <= N; j++) {
    double s = 0;
    for (int k = 0; k < N; k++) {
      const double th = M_PI * (k + 0.5) / N;
      const double y = a + (b - a) * (cos(th) + 1) / 2;
      s += cos(j * th) / y;
    }
    cf[j] = 2.0 * s / N;
  }
  float2 *v = arena(H, A_V), *tp = arena(H, A_TP), *tc = arena(H, A_TC), *ax = arena(H, A_AX),
         *tmp = arena(H, A_TMP), *hop = arena(H, A_HOP);
  int rc = hybrid_l1_apply(H, v, r, 1, 1, hop, st);
  if (rc == DWF_OK) rc = blas_axpby(c, 0.5 * cf[0], v, DWF_F32, 0.0, z, DWF_F32, n, st);
  if (rc || N < 2) return rc;
  const double xa = 2.0 / (b - a), xb = -(b + a) / (b - a);
  rc = blas_copy(c, tp, DWF_F32, v, DWF_F32, n, st);
  if (rc == DWF_OK) rc = hybrid_l1_apply(H, tmp, tp, 1, 1, hop, st);
  if (rc == DWF_OK) rc = hybrid_l1_apply(H, ax, tmp, 1, 1, hop, st);
  if (rc == DWF_OK) rc = blas_axpbypcz(c, xa, ax, xb, tp, 0.0, tc, n, DWF_F32, st);
  if (rc == DWF_OK) rc = blas_axpby(c, cf[1], tc, DWF_F32, 1.0, z, DWF_F32, n, st);
  for (int j = 2; j < N && rc == DWF_OK; j++) {
    rc = hybrid_l1_apply(H, tmp, tc, 1, 1, hop, st);
    if (rc == DWF_OK) rc = hybrid_l1_apply(H, ax, tmp, 1, 1, hop, st);
    if (rc == DWF_OK) rc = blas_cheb_step(c, tp, ax, tc, 2 * xa, 2 * xb, z, cf[j], n, DWF_F32, st);
    float2* t = tp;
    tp = tc;
    tc = t;
  }
  return rc;
}

// The level-2 solve of A_2 e = r (CG on A_2^2, red-black CG, or CG from the
// deflation guess, as the parameters choose).
int l2_solve(dwf_hybrid* H, float2* e, const float2* r, cudaStream_t st, int* ncoarse) {
  int it = 0;
  const int rc = H->p.coarse_solver == DWF_COARSE_RB
                     ? coarse_rbcg(H->C2, e, r, H->p.coarse_tol, H->p.coarse_maxiter, &it, st)
                     : coarse_cg(H->C2, e, r, H->p.coarse_tol, H->p.coarse_maxiter, &it, st);
  *ncoarse += it;
  return rc;
}

// Level-1 V(1,1) (Eqs. 26-28 with M = H_1) on one vector: smoother (when its
// order is not 0), coarse-coarse correction P2 A_2^-1 P2^dag, smoother.
int l1_vcycle(dwf_hybrid* H, float2* x, const float2* r, cudaStream_t st, int* ncoarse) {
  dwf_ctx* c = H->ctx;
  const int64_t n = n1(H);
  const bool smooth = H->hp.smooth1_order > 0;
  float2 *rr = arena(H, A_RR), *s2 = arena(H, A_S2), *hop = arena(H, A_HOP);
  float2* rc2 = (float2*)H->w[HW_L2];
  float2* ec2 = rc2 + (size_t)H->nc1 * H->nb2;
  int rc = DWF_OK;
  const float2* r1 = r;
  if (smooth) {
    rc = l1_smoother(H, x, r, st);
    if (rc == DWF_OK) rc = hybrid_l1_apply(H, rr, x, 1, 1, hop, st);
    if (rc == DWF_OK) rc = blas_axpby(c, 1.0, r, DWF_F32, -1.0, rr, DWF_F32, n, st);
    r1 = rr;
  }
  if (rc == DWF_OK) rc = hybrid_restrict2(H, rc2, r1, st);
  if (rc == DWF_OK) rc = l2_solve(H, ec2, rc2, st, ncoarse);
  if (rc == DWF_OK) rc = hybrid_prolong2(H, x, ec2, smooth ? 1 : 0, st);
  if (rc || !smooth) return rc;
  rc = hybrid_l1_apply(H, rr, x, 1, 1, hop, st);
  if (rc == DWF_OK) rc = blas_axpby(c, 1.0, r, DWF_F32, -1.0, rr, DWF_F32, n, st);
  if (rc == DWF_OK) rc = l1_smoother(H, s2, rr, st);
  if (rc == DWF_OK) rc = blas_axpby(c, 1.0, s2, DWF_F32, 1.0, x, DWF_F32, n, st);
  return rc;
}

// kcycle iterations of flexible GCR on H_1 e = r from e = 0, no tolerance test.
int l1_solve(dwf_hybrid* H, float2* e, const float2* r, cudaStream_t st, int* ncoarse) {
  dwf_ctx* c = H->ctx;
  const int64_t n = n1(H);
  const int K = H->hp.kcycle;
  float2 *res = arena(H, A_RES), *hop = arena(H, A_HOP);
  DWF_CUDA(c, cudaMemsetAsync(e, 0, n * sizeof(float2), st));
  int rc = norm2_dev(c, r, n, DWF_F32, S_TMP2, st);
  if (rc == DWF_OK) rc = read_scalars(c, S_TMP2, 1, st);
  if (rc) return rc;
  if (!(c->hscal[S_TMP2] > 0)) return isfinite(c->hscal[S_TMP2]) ? DWF_OK : dwf_fail(c, DWF_ENAN, "level-1 source");
  rc = blas_copy(c, res, DWF_F32, r, DWF_F32, n, st);
  std::vector<double> wn(K);
  for (int k = 0; k < K && rc == DWF_OK; k++) {
    float2* z = arena(H, A_ZW + k);
    float2* w = arena(H, A_ZW + K + k);
    rc = l1_vcycle(H, z, res, st, ncoarse);
    if (rc == DWF_OK) rc = hybrid_l1_apply(H, w, z, 1, 1, hop, st);
    for (int j = 0; j < k && rc == DWF_OK; j++) {
      const float2* wj = arena(H, A_ZW + K + j);
      const float2* zj = arena(H, A_ZW + j);
      int np = 0;
      rc = blas_cdot_partials(c, wj, w, n, DWF_F32, st, &np);
      if (rc == DWF_OK) rc = blas_finalize(c, np, 2, S_TMP0, st);
      if (rc == DWF_OK) rc = read_scalars(c, S_TMP0, 2, st);
      if (rc) break;
      const double br = c->hscal[S_TMP0] / wn[j], bi = c->hscal[S_TMP0 + 1] / wn[j];
      rc = blas_caxpy(c, -br, -bi, wj, DWF_F32, w, DWF_F32, n, st);
      if (rc == DWF_OK) rc = blas_caxpy(c, -br, -bi, zj, DWF_F32, z, DWF_F32, n, st);
    }
    if (rc) break;
    int np = 0;
    rc = blas_cdot_partials(c, w, res, n, DWF_F32, st, &np);
    if (rc == DWF_OK) rc = blas_finalize(c, np, 2, S_TMP0, st);
    if (rc == DWF_OK) rc = norm2_dev(c, w, n, DWF_F32, S_TMP2, st);
    if (rc == DWF_OK) rc = read_scalars(c, S_TMP0, 3, st);
    if (rc) break;
    const double ww = c->hscal[S_TMP2];
    if (!(ww > 0) || !isfinite(ww)) return dwf_fail(c, DWF_ENAN, "level-1 GCR breakdown");
    wn[k] = ww;
    const double ar = c->hscal[S_TMP0] / ww, ai = c->hscal[S_TMP0 + 1] / ww;
    rc = blas_caxpy(c, ar, ai, z, DWF_F32, e, DWF_F32, n, st);
    if (rc == DWF_OK && k + 1 < K) rc = blas_caxpy(c, -ar, -ai, w, DWF_F32, res, DWF_F32, n, st);
  }
  return rc;
}

}  // namespace

// The fine V-cycle's coarse correction: x += P1 e, e from the level-1 W-cycle
// solve of H_1 e = P1^dag r (FP32 full fields).
int hybrid_correction(dwf_hybrid* H, void* x, const void* r, cudaStream_t st, int* ncoarse) {
  int rc = arena_ready(H);
  if (rc) return rc;
  float2 *r1 = arena(H, A_R1), *e1 = arena(H, A_E1);
  rc = hybrid_restrict1(H, r1, (const float2*)r, 1, st);
  if (rc == DWF_OK) rc = l1_solve(H, e1, r1, st, ncoarse);
  if (rc == DWF_OK) rc = hybrid_prolong1(H, (float2*)x, e1, 1, 1, st);
  return rc;
}

int hybrid_level1_op(dwf_hybrid* H, int op, void* out, const void* in, int nvec, cudaStream_t st) {
  dwf_ctx* c = H->ctx;
  if (nvec < 1 || ((op >= 4) && nvec != 1) || ((op == 2 || op == 3) && nvec > 65535))
    return dwf_fail(c, DWF_EINVAL, "nvec");
  int rc = arena_ready(H);
  if (rc) return rc;
  switch (op) {
    case 0:
    case 1: {
      float2* tmp = (float2*)hws(H, HW_F4, (size_t)n1(H) * nvec * sizeof(float2));
      if (!tmp) return dwf_fail(c, DWF_ENOMEM, "hybrid workspace");
      return hybrid_l1_apply(H, (float2*)out, (const float2*)in, nvec, op, tmp, st);
    }
    case 2:
      return hybrid_restrict1(H, (float2*)out, (const float2*)in, nvec, st);
    case 3:
      return hybrid_prolong1(H, (float2*)out, (const float2*)in, nvec, 0, st);
    case 4:
      return hybrid_restrict2(H, (float2*)out, (const float2*)in, st);
    case 5:
      return hybrid_prolong2(H, (float2*)out, (const float2*)in, 0, st);
    case 6: {
      int nco = 0;
      rc = l1_solve(H, (float2*)out, (const float2*)in, st, &nco);
      if (rc) return rc;
      DWF_CUDA(c, cudaStreamSynchronize(st));
      return DWF_OK;
    }
    default:
      return dwf_fail(c, DWF_EINVAL, "bad level-1 operation");
  }
}

// ---------------------------------------------------------------------- setup
void hybrid_free(dwf_hybrid* H) {
  if (!H) return;
  if (H->phi64) cudaFree(H->phi64);
  if (H->phi32) cudaFree(H->phi32);
  if (H->Phi2) cudaFree(H->Phi2);
  if (H->C1) coarse_destroy(H->C1);
  if (H->C2) coarse_destroy(H->C2);
  for (int i = 0; i < 10; i++) hws_free(H, i);
  delete H;
}

namespace {

dwf_coarse* new_coarse(dwf_hybrid* H, int nb, int nplus, size_t* bytes64) {
  dwf_coarse* C = new (std::nothrow) dwf_coarse();
  if (!C) return nullptr;
  C->ctx = H->ctx;
  C->g = H->g;  // the level-1 lattice: Lc and nc of the 4D blocking
  C->nb = nb;
  C->nplus = nplus;
  const size_t na = (size_t)H->nc1 * 9 * nb * nb;
  *bytes64 = na;
  if (cudaMalloc(&C->A64, na * sizeof(double2)) != cudaSuccess || cudaMalloc(&C->A32, na * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    coarse_destroy(C);
    return nullptr;
  }
  return C;
}

// Steps 1-3 of the setup: the FP32 filter of the Gaussian 4D fields by
// T_order4(x(D_W^dag D_W)), the gamma_5 projection and block orthonormalisation
// in FP64, and the stencil B of -1/2 D_hop on the 4D basis.
int build_level1(dwf_hybrid* H, const void* eta4, cudaStream_t st) {
  dwf_ctx* c = H->ctx;
  const dwf_hybrid_params& hp = H->hp;
  dwf_ctx* c4 = nullptr;
  int rc = dwf_ctx_clone_ls(c, H->nb4, &c4, st);
  if (rc) return dwf_fail(c, rc, "4D basis context");
  const int64_t n4 = 2 * c->g.Vh * 12 * H->nb4;
  float2 *tp = (float2*)hws(H, HW_F0, n4 * sizeof(float2)), *tc = (float2*)hws(H, HW_F1, n4 * sizeof(float2)),
         *ax = (float2*)hws(H, HW_F2, n4 * sizeof(float2)), *tmp = (float2*)hws(H, HW_F3, n4 * sizeof(float2));
  if (!tp || !tc || !ax || !tmp || cudaMalloc(&H->phi64, n4 * sizeof(double2)) != cudaSuccess ||
      cudaMalloc(&H->phi32, n4 * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    dwf_ctx_destroy(c4);
    return dwf_fail(c, DWF_ENOMEM, "4D basis");
  }
  // D_W^dag D_W = (4+m)^2 Dh^dag Dh with Dh = 1 - kappa D_hop: the filter
  // interval scales by (4+m)^-2
  const double m4 = 4.0 + hp.mass4, kappa = 0.5 / m4, sc = m4 * m4;
  const double lo = hp.lambda_lo4 / sc, hi = hp.lambda_max4 / sc;
  const double a = 2.0 / (hi - lo), b = -(hi + lo) / (hi - lo);
  rc = blas_copy(c4, tp, DWF_F32, eta4, DWF_F64, n4, st);
  float2* res = tp;
  if (rc == DWF_OK && hp.order4 > 0) {
    rc = wilson_hat(c4, tmp, tp, kappa, 0, st, nullptr);
    if (rc == DWF_OK) rc = wilson_hat(c4, ax, tmp, kappa, 1, st, nullptr);
    if (rc == DWF_OK) rc = blas_axpbypcz(c4, a, ax, b, tp, 0.0, tc, n4, DWF_F32, st);  // T1
    for (int k = 2; k <= hp.order4 && rc == DWF_OK; k++) {
      const ChebFuse cf = {tc, tp, nullptr, 2 * a, 2 * b, 0.0};
      rc = wilson_hat(c4, tmp, tc, kappa, 0, st, nullptr);
      if (rc == DWF_OK) rc = wilson_hat(c4, nullptr, tmp, kappa, 1, st, &cf);  // tp <- T_k
      float2* t = tp;
      tp = tc;
      tc = t;
      if (rc == DWF_OK && k % 24 == 0) rc = rescale_pair(c4, tp, tc, n4, st);
    }
    res = tc;
  }
  if (rc == DWF_OK) rc = blas_copy(c4, H->phi64, DWF_F64, res, DWF_F32, n4, st);
  if (rc == DWF_OK) {
    c->launches++;
    hyb::k_chiral4<double2><<<nblk(n4), 256, 0, st>>>(H->phi64, n4, H->nb4, H->np4);
  }
  if (rc == DWF_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = dwf_cuda_check(c, e, "4D filter");
  }
  if (rc) {
    if (!c->err.size() && c4->err.size()) c->err = c4->err;
    dwf_ctx_destroy(c4);
    return rc;
  }
  rc = ortho4(H, st);
  if (rc == DWF_OK) rc = blas_copy(c, H->phi32, DWF_F32, H->phi64, DWF_F64, n4, st);
  // B[x][d] = Gram(phi, term d of -1/2 D_hop phi), FP64
  size_t na = 0;
  if (rc == DWF_OK) {
    H->C1 = new_coarse(H, H->nb4, H->np4, &na);
    if (!H->C1) rc = dwf_fail(c, DWF_ENOMEM, "level-1 stencil");
  }
  double2* W = rc == DWF_OK ? (double2*)hws(H, HW_F4, n4 * sizeof(double2)) : nullptr;
  if (rc == DWF_OK && !W) rc = dwf_fail(c, DWF_ENOMEM, "level-1 build workspace");
  for (int d = 0; d < 9 && rc == DWF_OK; d++) {
    c->launches += 2;
    hyb::k_hop4_part<<<nblk(n4 / 12, 128), 128, 0, st>>>(W, H->phi64, c->links64[0], c->links64[1], H->g4, H->nb4, d);
    hyb::k_gram4<<<(unsigned)H->nc1, 256, 0, st>>>(H->C1->A64 + (size_t)d * H->nb4 * H->nb4, 9LL * H->nb4 * H->nb4, H->phi64,
                                                   W, H->g4, H->nb4);
  }
  if (rc == DWF_OK) rc = blas_copy(c, H->C1->A32, DWF_F32, H->C1->A64, DWF_F64, (int64_t)na, st);
  if (rc == DWF_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = dwf_cuda_check(c, e, "level-1 build");
  }
  dwf_ctx_destroy(c4);
  for (int s = HW_F0; s <= HW_F4; s++) hws_free(H, s);
  return rc;
}

// Steps 4-6: the level-2 basis (FP32 filter of H_1^2 on the Gaussian level-1
// vectors, Gamma5_1 projection, per-site orthonormalisation) and the level-2
// stencil A2[x][d][i][j] = <Phi_i(x), Gamma5_1 (term d of M_1) Phi_j>.
int build_level2(dwf_hybrid* H, const void* eta1, cudaStream_t st) {
  dwf_ctx* c = H->ctx;
  const dwf_hybrid_params& hp = H->hp;
  const int nb = H->nb2;
  const int64_t nm = n1(H) * nb;  // one level-1 multi-vector of nb2 vectors
  if (cudaMalloc(&H->Phi2, nm * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    return dwf_fail(c, DWF_ENOMEM, "level-2 basis");
  }
  float2 *tp = H->Phi2, *tc = (float2*)hws(H, HW_F0, nm * sizeof(float2)),
         *ax = (float2*)hws(H, HW_F1, nm * sizeof(float2)), *tmp = (float2*)hws(H, HW_F2, nm * sizeof(float2)),
         *hop = (float2*)hws(H, HW_F3, nm * sizeof(float2));
  if (!tc || !ax || !tmp || !hop) return dwf_fail(c, DWF_ENOMEM, "level-2 filter workspace");
  int rc = blas_copy(c, tp, DWF_F32, eta1, DWF_F64, nm, st);
  const double lo = hp.lambda_lo1, hi = hp.lambda_max1;
  const double a = 2.0 / (hi - lo), b = -(hi + lo) / (hi - lo);
  float2* res = tp;
  if (rc == DWF_OK && hp.order1 > 0) {
    rc = hybrid_l1_apply(H, tmp, tp, nb, 1, hop, st);
    if (rc == DWF_OK) rc = hybrid_l1_apply(H, ax, tmp, nb, 1, hop, st);
    if (rc == DWF_OK) rc = blas_axpbypcz(c, a, ax, b, tp, 0.0, tc, nm, DWF_F32, st);
    for (int k = 2; k <= hp.order1 && rc == DWF_OK; k++) {
      rc = hybrid_l1_apply(H, tmp, tc, nb, 1, hop, st);
      if (rc == DWF_OK) rc = hybrid_l1_apply(H, ax, tmp, nb, 1, hop, st);
      if (rc == DWF_OK) rc = blas_cheb_step(c, tp, ax, tc, 2 * a, 2 * b, nullptr, 0.0, nm, DWF_F32, st);
      float2* t = tp;
      tp = tc;
      tc = t;
      if (rc == DWF_OK && k % 24 == 0) rc = rescale_pair(c, tp, tc, nm, st);
    }
    res = tc;
  }
  if (rc == DWF_OK && res != H->Phi2) rc = blas_copy(c, H->Phi2, DWF_F32, res, DWF_F32, nm, st);
  if (rc == DWF_OK) {
    const long long np = H->nc1 * H->nb4 * (H->Ls / 2) * nb;
    c->launches++;
    hyb::k_l1_chiral<<<nblk(np), 256, 0, st>>>(H->Phi2, H->nc1 * H->nb4, H->nb4, H->np4, H->Ls, nb, H->np2);
  }
  for (int s = HW_F0; s <= HW_F3; s++) hws_free(H, s);
  if (rc == DWF_OK) rc = ortho2(H, st);
  size_t na = 0;
  if (rc == DWF_OK) {
    H->C2 = new_coarse(H, nb, H->np2, &na);
    if (!H->C2) rc = dwf_fail(c, DWF_ENOMEM, "level-2 stencil");
  }
  double2* W = rc == DWF_OK ? (double2*)hws(H, HW_F4, nm * sizeof(double2)) : nullptr;
  if (rc == DWF_OK && !W) rc = dwf_fail(c, DWF_ENOMEM, "level-2 build workspace");
  const int nq = H->nb4 * H->Ls;
  for (int d = 0; d < 9 && rc == DWF_OK; d++) {
    c->launches += 2;
    hyb::k_dir_apply<<<nblk(nm), 256, 0, st>>>(W, H->Phi2, H->C1->A64, H->g.Lc[0], H->g.Lc[1], H->g.Lc[2], H->g.Lc[3],
                                               H->nb4, H->Ls * nb, d);
    if (d == 0) {
      c->launches++;
      hyb::k_l1_tail<double2, double2><<<nblk(nm), 256, 0, st>>>(W, W, H->Phi2, nm, H->nb4, H->np4, H->Ls, nb,
                                                                 5.0 - c->M5, H->p.mf, 0);
    }
    hyb::k_gram_site<double2><<<(unsigned)H->nc1, 256, 0, st>>>(H->C2->A64, 9LL * nb * nb, (long long)d * nb * nb,
                                                                 H->Phi2, W, nq, nb, 1, H->np4, H->Ls);
  }
  if (rc == DWF_OK) rc = blas_copy(c, H->C2->A32, DWF_F32, H->C2->A64, DWF_F64, (int64_t)na, st);
  if (rc == DWF_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = dwf_cuda_check(c, e, "level-2 build");
  }
  hws_free(H, HW_F4);
  return rc;
}

}  // namespace

int hybrid_build(dwf_ctx* c, const dwf_mg_params* p, const dwf_hybrid_params* hp, const void* eta4, const void* eta1,
                 dwf_hybrid** out, cudaStream_t st) {
  Timer timer;
  *out = nullptr;
  const int nb4 = hp->nbasis4, nb2 = hp->nbasis1;
  if (nb4 != 4 && nb4 != 8 && nb4 != 16 && nb4 != 24) return dwf_fail(c, DWF_EINVAL, "nbasis4 must be 4, 8, 16 or 24");
  if (nb2 < 2 || (nb2 & 1) || nb2 > 64) return dwf_fail(c, DWF_EINVAL, "nbasis1 must be even, <= 64");
  if (!(hp->mass4 > -4.0) || !(hp->lambda_max4 > hp->lambda_lo4) || !(hp->lambda_max1 > hp->lambda_lo1) ||
      hp->order4 < 0 || hp->order1 < 0 || hp->kcycle < 1 || hp->kcycle > 16 || hp->smooth1_order < 0 ||
      (hp->smooth1_order > 0 && !(hp->smooth1_hi > hp->smooth1_lo && hp->smooth1_lo > 0)))
    return dwf_fail(c, DWF_EINVAL, "bad hybrid parameters");
  // without a level-1 smoother the preconditioner K = P2 A_2^-1 P2^dag obeys
  // K H_1 K = K, so a second GCR direction would vanish
  if (hp->kcycle > 1 && hp->smooth1_order == 0)
    return dwf_fail(c, DWF_EINVAL, "kcycle > 1 needs a level-1 smoother");
  if (!dwf_is_device_ptr(eta4) || !dwf_is_device_ptr(eta1)) return dwf_fail(c, DWF_EINVAL, "eta4, eta1: device memory");
  dwf_hybrid* H = new (std::nothrow) dwf_hybrid();
  if (!H) return DWF_ENOMEM;
  H->ctx = c;
  H->p = *p;
  H->hp = *hp;
  int b4 = 1, nc = 1;
  for (int m = 0; m < 4; m++) {
    if (hp->block[m] < 1 || c->g.L[m] % hp->block[m]) {
      delete H;
      return dwf_fail(c, DWF_EINVAL, "block does not tile the lattice");
    }
    H->g.L[m] = c->g.L[m];
    H->g.b[m] = hp->block[m];
    H->g.Lc[m] = c->g.L[m] / hp->block[m];
    b4 *= hp->block[m];
    nc *= H->g.Lc[m];
  }
  H->g.Lxh = c->g.Lxh;
  H->g.Vh = (int)c->g.Vh;
  H->g.Ls = c->g.Ls;
  H->g.b4 = b4;
  H->g.nc = nc;
  H->g4 = H->g;
  H->g4.Ls = nb4;
  H->nb4 = nb4;
  H->np4 = nb4 / 2;
  H->nb2 = nb2;
  H->np2 = nb2 / 2;
  H->Ls = c->g.Ls;
  H->nc1 = nc;
  int rc = build_level1(H, eta4, st);
  H->setup_seconds = timer.sec();
  Timer t2;
  if (rc == DWF_OK) rc = build_level2(H, eta1, st);
  if (rc == DWF_OK && p->coarse_solver == DWF_COARSE_RB) rc = coarse_rb_ready(H->C2, st);
  if (rc == DWF_OK && p->coarse_solver == DWF_COARSE_DEFLATED) {
    // Lanczos start: the level-2 restriction of the first eta1 vector
    const int64_t nv1 = n1(H);
    double2* e64 = (double2*)hws(H, HW_F0, nv1 * sizeof(double2));
    float2* e32 = (float2*)hws(H, HW_F1, nv1 * sizeof(float2));
    float2* v0 = (float2*)hws(H, HW_F2, (size_t)H->nc1 * nb2 * sizeof(float2));
    if (!e64 || !e32 || !v0) rc = dwf_fail(c, DWF_ENOMEM, "deflation start");
    if (rc == DWF_OK) {
      c->launches++;
      hyb::k_column<<<nblk(nv1), 256, 0, st>>>(e64, (const double2*)eta1, nv1, nb2);
    }
    if (rc == DWF_OK) rc = blas_copy(c, e32, DWF_F32, e64, DWF_F64, nv1, st);
    if (rc == DWF_OK) rc = hybrid_restrict2(H, v0, e32, st);
    if (rc == DWF_OK)
      rc = coarse_deflate(H->C2, v0, p->coarse_nev, p->coarse_lanczos, p->coarse_cheb_order, p->coarse_cheb_lo, 0.0,
                          nullptr, st);
    for (int s = HW_F0; s <= HW_F2; s++) hws_free(H, s);
  }
  if (rc == DWF_OK) rc = arena_ready(H);
  if (rc == DWF_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = dwf_cuda_check(c, e, "hybrid setup");
  }
  for (int s = HW_F0; s <= HW_FAIL; s++) hws_free(H, s);
  H->coarse_op_seconds = t2.sec();
  if (rc) {
    hybrid_free(H);
    return rc;
  }
  *out = H;
  return DWF_OK;
}

dwf_coarse* hybrid_coarse(dwf_hybrid* H) { return H ? H->C2 : nullptr; }
double hybrid_setup_seconds(const dwf_hybrid* H) { return H->setup_seconds; }
double hybrid_coarse_seconds(const dwf_hybrid* H) { return H->coarse_op_seconds; }

int hybrid_export(const dwf_hybrid* H, int what, void* out) {
  const void* src = nullptr;
  size_t bytes = 0;
  switch (what) {
    case 0:
      src = H->phi64;
      bytes = (size_t)2 * H->ctx->g.Vh * 12 * H->nb4 * sizeof(double2);
      break;
    case 1:
      src = H->C1->A64;
      bytes = (size_t)H->nc1 * 9 * H->nb4 * H->nb4 * sizeof(double2);
      break;
    case 2:
      src = H->Phi2;
      bytes = (size_t)n1(H) * H->nb2 * sizeof(float2);
      break;
    case 3:
      src = H->C2->A64;
      bytes = (size_t)H->nc1 * 9 * H->nb2 * H->nb2 * sizeof(double2);
      break;
    default:
      return DWF_EINVAL;
  }
  if (cudaMemcpy(out, src, bytes, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return DWF_ECUDA;
  }
  return DWF_OK;
}
