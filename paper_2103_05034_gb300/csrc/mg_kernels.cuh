// Kernels of the HDCR coarsening (arXiv:2103.05034, Sec. 3.1 and Sec. 3.4):
// block geometry, chirality projection, block inner products (restriction,
// Gram matrices), block linear combinations (prolongation, Cholesky-QR
// updates), the face-split hopping term used to build the 9-point little
// Dirac operator, and the coarse stencil apply on CUDA cores.
#pragma once
#include "dhop_impl.cuh"
#include "dwf_internal.cuh"

namespace dwfmg {

// Geometry of a blocking: fine lattice L, block b (spanning all of Ls), coarse Lc.
struct BlockGeom {
  int L[4], b[4], Lc[4];
  int Lxh, Vh, Ls;
  int b4;   // sites per block
  int nc;   // coarse sites
};

// Offset (in complex numbers, within one full field) of the Ls x 12 row of the
// i-th site of block xc, and whether it lies on the face of direction d (d = 0:
// always true; d = 1+2mu: the +mu face; d = 2+2mu: the -mu face).
__device__ __forceinline__ long long block_site_offset(const BlockGeom& g, int xc, int i, int d,
                                                       bool* on_face) {
  int cc[4], ii[4];
  int r = xc;
  cc[0] = r % g.Lc[0];
  r /= g.Lc[0];
  cc[1] = r % g.Lc[1];
  r /= g.Lc[1];
  cc[2] = r % g.Lc[2];
  cc[3] = r / g.Lc[2];
  r = i;
  ii[0] = r % g.b[0];
  r /= g.b[0];
  ii[1] = r % g.b[1];
  r /= g.b[1];
  ii[2] = r % g.b[2];
  ii[3] = r / g.b[2];
  int x[4];
#pragma unroll
  for (int m = 0; m < 4; m++) x[m] = cc[m] * g.b[m] + ii[m];
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  const long long lex = x[0] + (long long)g.L[0] * (x[1] + (long long)g.L[1] * (x[2] + (long long)g.L[2] * x[3]));
  if (d == 0) {
    *on_face = true;
  } else {
    const int mu = (d - 1) >> 1;
    const bool fwd = ((d - 1) & 1) == 0;
    *on_face = fwd ? (ii[mu] == g.b[mu] - 1) : (ii[mu] == 0);
  }
  return ((long long)p * g.Vh + (lex >> 1)) * 12LL * g.Ls;
}

// Coarse neighbour of xc in direction d (periodic).
__device__ __forceinline__ int coarse_nbr(const int Lc[4], int xc, int d) {
  if (d == 0) return xc;
  int c[4];
  int r = xc;
  c[0] = r % Lc[0];
  r /= Lc[0];
  c[1] = r % Lc[1];
  r /= Lc[1];
  c[2] = r % Lc[2];
  c[3] = r / Lc[2];
  const int mu = (d - 1) >> 1;
  const bool fwd = ((d - 1) & 1) == 0;
  c[mu] = fwd ? (c[mu] + 1 == Lc[mu] ? 0 : c[mu] + 1) : (c[mu] == 0 ? Lc[mu] - 1 : c[mu] - 1);
  return c[0] + Lc[0] * (c[1] + Lc[1] * (c[2] + Lc[2] * c[3]));
}

// (1 + sign Gamma_5)/2 on full fields: (Gamma_5 psi)_s = gamma_5 psi_{Ls-1-s}.
template <int P>
__global__ void k_chiral_project(typename Prec<P>::S* out, const typename Prec<P>::S* in, long long n,
                                 int Ls, float sign) {
  typedef typename Prec<P>::R R;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const long long row = e / Ls;
  const int s = (int)(e - row * Ls);
  const int c = (int)(row % 12);
  const R g = (c < 6) ? R(sign) : R(-sign);
  const auto a = ld_c(in + e);
  const auto b = ld_c(in + row * Ls + (Ls - 1 - s));
  cpx<R> o;
  o.re = R(0.5) * (a.re + g * b.re);
  o.im = R(0.5) * (a.im + g * b.im);
  st_c(out + e, o);
}

// out[xc][j][k] (+)= sum over the sites of block xc (on the face of d) and all
// (s, spin, colour) of conj(X_j) Y_k.  nx, ny <= 32 per CTA tile; FP64 sums of
// 16-element partial sums in the storage's arithmetic type.
constexpr int BI_CH = 16;
template <int P>
__global__ void __launch_bounds__(256) k_block_inner(const typename Prec<P>::S* X, long long xstride, int nx,
                                                     const typename Prec<P>::S* Y, long long ystride, int ny,
                                                     double2* out, long long out_bstride, int out_ld,
                                                     BlockGeom g, int d, int accumulate) {
  typedef typename Prec<P>::R R;
  __shared__ cpx<R> sx[32][BI_CH + 1];
  __shared__ cpx<R> sy[32][BI_CH + 1];
  const int xc = blockIdx.x;
  const int j0 = blockIdx.y * 32, k0 = blockIdx.z * 32;
  const int nj = min(32, nx - j0), nk = min(32, ny - k0);
  const int tid = threadIdx.x;
  double2 acc[4];
#pragma unroll
  for (int q = 0; q < 4; q++) acc[q] = make_double2(0, 0);
  const int row_len = 12 * g.Ls;
  for (int i = 0; i < g.b4; i++) {
    bool face;
    const long long off = block_site_offset(g, xc, i, d, &face);
    if (!face) continue;
    for (int ch = 0; ch < row_len; ch += BI_CH) {
      for (int e = tid; e < 32 * BI_CH; e += 256) {
        const int v = e / BI_CH, q = e - v * BI_CH;
        sx[v][q] = v < nj ? ld_c(X + (j0 + v) * xstride + off + ch + q) : cmake<R>(0, 0);
        sy[v][q] = v < nk ? ld_c(Y + (k0 + v) * ystride + off + ch + q) : cmake<R>(0, 0);
      }
      __syncthreads();
#pragma unroll
      for (int qq = 0; qq < 4; qq++) {
        const int ent = tid + 256 * qq;
        const int j = ent >> 5, k = ent & 31;
        R re = 0, im = 0;
#pragma unroll
        for (int q = 0; q < BI_CH; q++) {
          const cpx<R> a = sx[j][q], b = sy[k][q];
          re = fma(a.re, b.re, re);
          re = fma(a.im, b.im, re);
          im = fma(a.re, b.im, im);
          im = fma(-a.im, b.re, im);
        }
        acc[qq].x += (double)re;
        acc[qq].y += (double)im;
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int qq = 0; qq < 4; qq++) {
    const int ent = tid + 256 * qq;
    const int j = ent >> 5, k = ent & 31;
    if (j < nj && k < nk) {
      double2* o = out + xc * out_bstride + (long long)(j0 + j) * out_ld + (k0 + k);
      if (accumulate) {
        o->x += acc[qq].x;
        o->y += acc[qq].y;
      } else {
        *o = acc[qq];
      }
    }
  }
}

// Restriction of one field: out[xc][j] = sum over block xc of conj(X_j) Y,
// for nx <= 64 basis fields (the Gram-matrix kernel above would compute 32
// columns of which one is wanted).  One CTA per block, eight warps; warp w
// owns the basis fields j = w*J .. w*J+J-1 (J = NX/8) and walks all of the
// block's elements with its 32 lanes (coalesced), so every basis element is
// read once; sums of 16 terms in the storage's arithmetic type are added in
// FP64 and reduced across the warp in FP64.
template <int P, int NX>
__global__ void __launch_bounds__(256) k_block_restrict(const typename Prec<P>::S* X, long long xstride, int nx,
                                                        const typename Prec<P>::S* Y, double2* out,
                                                        long long out_bstride, int out_ld, BlockGeom g) {
  typedef typename Prec<P>::R R;
  constexpr int J = NX / 8;
  const int xc = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int j0 = w * J;
  double2 acc[J];
  cpx<R> part[J];
#pragma unroll
  for (int j = 0; j < J; j++) {
    acc[j] = make_double2(0, 0);
    part[j] = cmake<R>(0, 0);
  }
  const int row_len = 12 * g.Ls;
  const int nel = g.b4 * row_len;
  int cnt = 0;
  for (int e = lane; e < nel; e += 32) {
    const int i = e / row_len, q = e - i * row_len;
    bool face;
    const long long off = block_site_offset(g, xc, i, 0, &face) + q;
    const cpx<R> y = ld_c(Y + off);
#pragma unroll
    for (int j = 0; j < J; j++) {
      if (j0 + j < nx) {
        const cpx<R> a = ld_c(X + (long long)(j0 + j) * xstride + off);
        part[j].re = fma(a.re, y.re, part[j].re);
        part[j].re = fma(a.im, y.im, part[j].re);
        part[j].im = fma(a.re, y.im, part[j].im);
        part[j].im = fma(-a.im, y.re, part[j].im);
      }
    }
    if (++cnt == 16) {
      cnt = 0;
#pragma unroll
      for (int j = 0; j < J; j++) {
        acc[j].x += (double)part[j].re;
        acc[j].y += (double)part[j].im;
        part[j] = cmake<R>(0, 0);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < J; j++) {
    double x = acc[j].x + (double)part[j].re, y = acc[j].y + (double)part[j].im;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_down_sync(0xffffffffu, x, o);
      y += __shfl_down_sync(0xffffffffu, y, o);
    }
    if (lane == 0 && j0 + j < nx) out[xc * out_bstride + (long long)(j0 + j) * out_ld] = make_double2(x, y);
  }
}

// Y_k(site) = sum_j X_j(site) M[xc][j][k] over every site of every block:
// prolongation (M = coarse vector) and Cholesky-QR updates (M = R^-1).
// One CTA per block; M staged in shared memory (nx * ny <= 1024).
// The arithmetic is FP64 when either side is stored in FP64 (the Gram-Schmidt
// of the basis), FP32 otherwise (prolongation inside the V-cycle).
template <int PX, int PY>
__global__ void __launch_bounds__(256) k_block_combine(typename Prec<PY>::S* Y, long long ystride, int ny,
                                                       const typename Prec<PX>::S* X, long long xstride,
                                                       int nx, const double2* M, long long m_bstride,
                                                       int m_ld, BlockGeom g, int accumulate) {
  typedef typename Prec<PY>::R RY;
  typedef typename std::conditional<PX == DWF_F64 || PY == DWF_F64, double, float>::type RC;
  __shared__ cpx<RC> sm[1024];
  const int xc = blockIdx.x;
  for (int e = threadIdx.x; e < nx * ny; e += blockDim.x) {
    const int j = e / ny, k = e - j * ny;
    const double2 m = M[xc * m_bstride + (long long)j * m_ld + k];
    sm[e] = cmake<RC>((RC)m.x, (RC)m.y);
  }
  __syncthreads();
  const int row_len = 12 * g.Ls;
  const int nel = g.b4 * row_len;
  for (int e = threadIdx.x; e < nel; e += blockDim.x) {
    const int i = e / row_len, q = e - i * row_len;
    bool face;
    const long long off = block_site_offset(g, xc, i, 0, &face) + q;
    for (int k = 0; k < ny; k++) {
      RC re = 0, im = 0;
      for (int j = 0; j < nx; j++) {
        const auto v = ld_c(X + j * xstride + off);
        const cpx<RC> m = sm[j * ny + k];
        re = fma((RC)v.re, m.re, re);
        re = fma(-(RC)v.im, m.im, re);
        im = fma((RC)v.re, m.im, im);
        im = fma((RC)v.im, m.re, im);
      }
      typename Prec<PY>::S* yp = Y + k * ystride + off;
      if (accumulate) {
        const auto yv = ld_c(yp);
        re += (RC)yv.re;
        im += (RC)yv.im;
      }
      st_c(yp, cmake<RY>((RY)re, (RY)im));
    }
  }
}

// In-place form of the Cholesky-QR update for a group of n <= 32 FP32 fields
// (x_k <- sum_{j <= k} x_j Rinv[xc][j][k], Rinv upper triangular within the
// group, rows and columns offset by g0 in the nb x nb matrix): each thread
// owns one element of the block, reads it from all n fields first and then
// writes the n results, so no second copy of the basis is needed.  FP32
// arithmetic, the precision the fields are stored in (the Gram matrices and
// their factorisation, which decide the result's orthogonality, stay FP64).
static __global__ void __launch_bounds__(256) k_block_update_inplace(float2* X, long long xstride, int n, int g0, int nb,
                                                              const double2* Rinv, BlockGeom g) {
  __shared__ float2 sm[32 * 32];
  const int xc = blockIdx.x;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int j = e / n, k = e - j * n;
    const double2 r = Rinv[(long long)xc * nb * nb + (long long)(g0 + j) * nb + g0 + k];
    sm[e] = make_float2((float)r.x, (float)r.y);
  }
  __syncthreads();
  const int row_len = 12 * g.Ls;
  const int nel = g.b4 * row_len;
  for (int e = threadIdx.x; e < nel; e += blockDim.x) {
    const int i = e / row_len, q = e - i * row_len;
    bool face;
    const long long off = block_site_offset(g, xc, i, 0, &face) + q;
    float2 v[32];
#pragma unroll
    for (int j = 0; j < 32; j++)
      if (j < n) v[j] = X[(long long)j * xstride + off];
#pragma unroll
    for (int k = 0; k < 32; k++) {
      if (k >= n) break;
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int j = 0; j < 32; j++) {
        if (j > k) break;
        const float2 m = sm[j * n + k];
        re = fmaf(v[j].x, m.x, re);
        re = fmaf(-v[j].y, m.y, re);
        im = fmaf(v[j].x, m.y, im);
        im = fmaf(v[j].y, m.x, im);
      }
      X[(long long)k * xstride + off] = make_float2(re, im);
    }
  }
}

// Cholesky G = R^dag R of each (block, group) Gram sub-matrix and R^-1 written
// into Rinv[xc][j][k] (upper triangular within the group; entries across groups
// are left untouched, so Rinv must be zeroed first).  One CTA per (block,
// group); thread 0 factorises in shared memory (groups of at most 32 vectors).
// Sets *fail if a pivot is not positive (the vectors are linearly dependent on
// that block).
// shift_rel > 0 factorises G + shift_rel * max_k G_kk * 1 instead (the first
// pass of shifted Cholesky-QR for vectors stored in FP32, whose Gram matrices
// may be numerically singular).
static __global__ void k_block_cholinv(const double2* G, double2* Rinv, int nb, int nplus, int* fail,
                                       double shift_rel = 0.0) {
  __shared__ double2 R[32][33];
  __shared__ double2 Ri[32][33];
  const int xc = blockIdx.x, grp = blockIdx.y;
  const int g0 = grp ? nplus : 0, n = grp ? nb - nplus : nplus;
  if (n <= 0 || n > 32 || threadIdx.x != 0) return;
  const double2* Gb = G + (long long)xc * nb * nb;
  double2* Rb = Rinv + (long long)xc * nb * nb;
  for (int a = 0; a < n; a++)
    for (int b = 0; b < n; b++) {
      R[a][b] = make_double2(0, 0);
      Ri[a][b] = make_double2(0, 0);
    }
  double shift = 0.0;
  if (shift_rel > 0) {
    for (int k = 0; k < n; k++) shift = fmax(shift, Gb[(g0 + k) * nb + g0 + k].x);
    shift *= shift_rel;
  }
  for (int k = 0; k < n; k++) {
    double dkk = Gb[(g0 + k) * nb + g0 + k].x + shift;
    for (int i = 0; i < k; i++) dkk -= R[i][k].x * R[i][k].x + R[i][k].y * R[i][k].y;
    if (!(dkk > 0)) {
      atomicExch(fail, 1);
      return;
    }
    const double rkk = sqrt(dkk);
    R[k][k] = make_double2(rkk, 0);
    for (int j = k + 1; j < n; j++) {
      double2 v = Gb[(g0 + k) * nb + g0 + j];
      for (int i = 0; i < k; i++) {  // v -= conj(R_ik) R_ij
        v.x -= R[i][k].x * R[i][j].x + R[i][k].y * R[i][j].y;
        v.y -= R[i][k].x * R[i][j].y - R[i][k].y * R[i][j].x;
      }
      R[k][j] = make_double2(v.x / rkk, v.y / rkk);
    }
  }
  for (int k = 0; k < n; k++) {  // rows of R^-1
    Ri[k][k] = make_double2(1.0 / R[k][k].x, 0);
    for (int j = k + 1; j < n; j++) {
      double re = 0, im = 0;
      for (int i = k; i < j; i++) {
        re += Ri[k][i].x * R[i][j].x - Ri[k][i].y * R[i][j].y;
        im += Ri[k][i].x * R[i][j].y + Ri[k][i].y * R[i][j].x;
      }
      const double rjj = R[j][j].x;
      Ri[k][j] = make_double2(-re / rjj, -im / rjj);
    }
  }
  for (int a = 0; a < n; a++)
    for (int b = 0; b < n; b++) Rb[(g0 + a) * nb + g0 + b] = Ri[a][b];
}

// One term of H_DW = Gamma_5 D_DW that crosses a block face: for d = 1+2mu
// (2+2mu) the hop from x+mu (x-mu), -1/2 (1 -+ gamma_mu) U psi, kept only at
// sites on the +mu (-mu) face of their block, then Gamma_5.  Full fields.
template <int P, int LS>
__global__ void __launch_bounds__(128) k_face_hop(typename Prec<P>::S* out, const typename Prec<P>::S* in,
                                                  long long rhs_stride, const typename Prec<P>::LS* links0,
                                                  const typename Prec<P>::LS* links1, BlockGeom g, int d) {
  typedef typename Prec<P>::R R;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (parity, site, s)
  const int rhs = blockIdx.y;
  const long long nsite5 = 2LL * g.Vh * LS;
  if (e >= nsite5) return;
  const int s = (int)(e % LS);
  const long long ps = e / LS;
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
  const int mu = (d - 1) >> 1;
  const bool fwd = ((d - 1) & 1) == 0;
  const bool face = fwd ? (x[mu] % g.b[mu] == g.b[mu] - 1) : (x[mu] % g.b[mu] == 0);
  typename Prec<P>::S* o = out + rhs * rhs_stride + ps * 12 * LS;
  if (!face) {
#pragma unroll
    for (int c = 0; c < 12; c++) st_c(o + c * LS + s, cmake<R>(0, 0));
    return;
  }
  int y[4] = {x[0], x[1], x[2], x[3]};
  y[mu] = fwd ? (y[mu] + 1 == g.L[mu] ? 0 : y[mu] + 1) : (y[mu] == 0 ? g.L[mu] - 1 : y[mu] - 1);
  const long long ylex = y[0] + (long long)g.L[0] * (y[1] + (long long)g.L[1] * (y[2] + (long long)g.L[2] * y[3]));
  const typename Prec<P>::S* src = in + rhs * rhs_stride + ((long long)(1 - p) * g.Vh + (ylex >> 1)) * 12 * LS;
  cpx<R> ps12[12], acc[12];
#pragma unroll
  for (int c = 0; c < 12; c++) {
    ps12[c] = ld_c(src + c * LS + s);
    acc[c] = cmake<R>(0, 0);
  }
  cpx<R> U[9];
  const typename Prec<P>::LS* lk = (p ? links1 : links0) + ((long long)h * 8 + 2 * mu + (fwd ? 0 : 1)) * 9;
#pragma unroll
  for (int a = 0; a < 9; a++) U[a] = cmake<R>((R)lk[a].x, (R)lk[a].y);
  const R sg = fwd ? R(1) : R(-1);
  switch (mu) {
    case 0:
      dwfk::hop_dir<R, 0>(acc, ps12, U, sg);
      break;
    case 1:
      dwfk::hop_dir<R, 1>(acc, ps12, U, sg);
      break;
    case 2:
      dwfk::hop_dir<R, 2>(acc, ps12, U, sg);
      break;
    default:
      dwfk::hop_dir<R, 3>(acc, ps12, U, sg);
      break;
  }
  const int so = LS - 1 - s;
#pragma unroll
  for (int c = 0; c < 12; c++) {
    const R f = c < 6 ? R(-0.5) : R(0.5);  // -1/2 and gamma_5
    st_c(o + c * LS + so, cmake<R>(f * acc[c].re, f * acc[c].im));
  }
}

// Coarse 9-point stencil on CUDA cores: out[x][j][r] = sum_d sum_k
// A[x][d][j][k] in[x+d][k][r]; vectors [nc][nb][nrhs] complex FP32.
// One thread per output (site x, row j, right-hand side r); threads of a warp
// share x and j (broadcast A element) and read consecutive r (coalesced).
// NB > 0 fixes nb at compile time so that the k loop unrolls and its loads
// are all in flight together.
template <int NB>
__global__ void __launch_bounds__(256) k_coarse_apply(float2* out, const float2* in, const float2* A, int Lc0,
                                                      int Lc1, int Lc2, int Lc3, int nb_rt, int nrhs) {
  const int nb = NB > 0 ? NB : nb_rt;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = Lc0 * Lc1 * Lc2 * Lc3;
  if (e >= (long long)nc * nb * nrhs) return;
  const int r = (int)(e % nrhs);
  const long long t = e / nrhs;
  const int j = (int)(t % nb);
  const int x = (int)(t / nb);
  const int Lc[4] = {Lc0, Lc1, Lc2, Lc3};
  float re = 0.f, im = 0.f, re2 = 0.f, im2 = 0.f;
  for (int d = 0; d < 9; d++) {
    const int y = coarse_nbr(Lc, x, d);
    const float2* Ad = A + (((long long)x * 9 + d) * nb + j) * nb;
    const float2* v = in + (long long)y * nb * nrhs + r;
#pragma unroll
    for (int k = 0; k < (NB > 0 ? NB : 1); k += 2) {
      if (NB == 0) break;
      const float2 a = __ldg(Ad + k), a2 = __ldg(Ad + k + 1);
      const float2 b = __ldg(v + (long long)k * nrhs), b2 = __ldg(v + (long long)(k + 1) * nrhs);
      re = fmaf(a.x, b.x, re);
      re = fmaf(-a.y, b.y, re);
      im = fmaf(a.x, b.y, im);
      im = fmaf(a.y, b.x, im);
      re2 = fmaf(a2.x, b2.x, re2);
      re2 = fmaf(-a2.y, b2.y, re2);
      im2 = fmaf(a2.x, b2.y, im2);
      im2 = fmaf(a2.y, b2.x, im2);
    }
    if (NB == 0) {
      for (int k = 0; k < nb; k++) {
        const float2 a = Ad[k];
        const float2 b = v[(long long)k * nrhs];
        re = fmaf(a.x, b.x, re);
        re = fmaf(-a.y, b.y, re);
        im = fmaf(a.x, b.y, im);
        im = fmaf(a.y, b.x, im);
      }
    }
  }
  out[e] = make_float2(re + re2, im + im2);
}

// The same stencil with four consecutive right-hand sides per thread (nrhs a
// multiple of 4, vectors 16-byte aligned): each operator element feeds four
// outputs and the vector loads are 16-byte, so the kernel issues 0.75 loads
// per complex multiply-add instead of 2 (used below 32 right-hand sides).
template <int NB>
__global__ void __launch_bounds__(256) k_coarse_apply4(float2* out, const float2* in, const float2* A, int Lc0,
                                                       int Lc1, int Lc2, int Lc3, int nb_rt, int nrhs) {
  const int nb = NB > 0 ? NB : nb_rt;
  const int nq = nrhs >> 2;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = Lc0 * Lc1 * Lc2 * Lc3;
  if (e >= (long long)nc * nb * nq) return;
  const int q = (int)(e % nq);
  const long long t = e / nq;
  const int j = (int)(t % nb);
  const int x = (int)(t / nb);
  const int Lc[4] = {Lc0, Lc1, Lc2, Lc3};
  float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int d = 0; d < 9; d++) {
    const int y = coarse_nbr(Lc, x, d);
    const float2* Ad = A + (((long long)x * 9 + d) * nb + j) * nb;
    const float4* v = (const float4*)(in + (long long)y * nb * nrhs) + 2 * q;
#pragma unroll 4
    for (int k = 0; k < (NB > 0 ? NB : nb); k++) {
      const float2 a = __ldg(Ad + k);
      const float4 b0 = __ldg(v + (long long)k * (nrhs >> 1)), b1 = __ldg(v + (long long)k * (nrhs >> 1) + 1);
      acc0.x = fmaf(a.x, b0.x, acc0.x);
      acc0.x = fmaf(-a.y, b0.y, acc0.x);
      acc0.y = fmaf(a.x, b0.y, acc0.y);
      acc0.y = fmaf(a.y, b0.x, acc0.y);
      acc0.z = fmaf(a.x, b0.z, acc0.z);
      acc0.z = fmaf(-a.y, b0.w, acc0.z);
      acc0.w = fmaf(a.x, b0.w, acc0.w);
      acc0.w = fmaf(a.y, b0.z, acc0.w);
      acc1.x = fmaf(a.x, b1.x, acc1.x);
      acc1.x = fmaf(-a.y, b1.y, acc1.x);
      acc1.y = fmaf(a.x, b1.y, acc1.y);
      acc1.y = fmaf(a.y, b1.x, acc1.y);
      acc1.z = fmaf(a.x, b1.z, acc1.z);
      acc1.z = fmaf(-a.y, b1.w, acc1.z);
      acc1.w = fmaf(a.x, b1.w, acc1.w);
      acc1.w = fmaf(a.y, b1.z, acc1.w);
    }
  }
  float4* o = (float4*)(out + ((long long)x * nb + j) * nrhs) + 2 * q;
  o[0] = acc0;
  o[1] = acc1;
}

}  // namespace dwfmg
