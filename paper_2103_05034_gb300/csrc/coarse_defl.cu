// Coarse-space deflation (Sec. 3.5: eigenvector deflation of the coarse
// operator, the eigenvectors from a Lanczos run on a Chebyshev polynomial of
// the operator).  The paper gives no more detail; this follows the reading
// stated in the library's design notes:
//   * Lanczos with full reorthogonalisation on B = T_n(y(A^2)),
//     y(t) = 2 (t - lam_lo) / (lam_max - lam_lo) - 1, n even, so that the modes
//     of A^2 below lam_lo are B's largest; nk steps from the caller's start
//     vector;
//   * the nev Ritz vectors of T's largest eigenvalues are diagonalised with A^2
//     itself (Rayleigh-Ritz), giving pairs (theta_i, v_i);
//   * the coarse CG on A^2 then starts from x0 = sum_i v_i <v_i, A r> / theta_i.
// The vectors are FP32 coarse fields [nc][nb] (the precision of the coarse
// solve), inner products in FP64; the small dense eigenproblems (the nk x nk
// tridiagonal matrix and the nev x nev Rayleigh-Ritz matrix) are solved on the
// host by the cyclic Jacobi method for hermitian matrices.
#include <math.h>
#include <string.h>

#include <complex>
#include <vector>

#include "coarse_internal.cuh"

namespace {

constexpr int DT = 256;

// out[q] = scale[q] * sum_i conj(Q[q][i]) w[i] for q < nq (one CTA per q,
// FP64 sums in a fixed order); scale may be null.
__global__ void __launch_bounds__(DT) k_multidot(const float2* __restrict__ Q, long long ld, const float2* __restrict__ w,
                                                 long long n, double2* out, const double* scale) {
  __shared__ double sr[DT / 32], si[DT / 32];
  const int q = blockIdx.x;
  const float2* Qq = Q + (size_t)q * ld;
  double re = 0.0, im = 0.0;
  for (long long i = threadIdx.x; i < n; i += DT) {
    const float2 a = Qq[i], b = w[i];
    re += (double)a.x * b.x + (double)a.y * b.y;
    im += (double)a.x * b.y - (double)a.y * b.x;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = re;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < DT / 32; k++) {
      a += sr[k];
      b += si[k];
    }
    const double f = scale ? scale[q] : 1.0;
    out[q] = make_double2(a * f, b * f);
  }
}

// w[i] = alpha w[i] + sgn * sum_q Q[q][i] c[q] (FP64 sum per element).
__global__ void __launch_bounds__(DT) k_multicomb(float2* w, const float2* __restrict__ Q, long long ld, int nq,
                                                  long long n, const double2* __restrict__ c, float alpha, double sgn) {
  for (long long i = (long long)blockIdx.x * DT + threadIdx.x; i < n; i += (long long)gridDim.x * DT) {
    double re = 0.0, im = 0.0;
    for (int q = 0; q < nq; q++) {
      const float2 a = Q[(size_t)q * ld + i];
      const double2 b = c[q];
      re += a.x * b.x - a.y * b.y;
      im += a.x * b.y + a.y * b.x;
    }
    const float2 o = alpha == 0.f ? make_float2(0.f, 0.f) : w[i];
    w[i] = make_float2((float)(alpha * o.x + sgn * re), (float)(alpha * o.y + sgn * im));
  }
}

unsigned comb_grid(long long n) {
  long long g = (n + DT - 1) / DT;
  return (unsigned)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

typedef std::complex<double> cd;

// Cyclic Jacobi for a hermitian n x n matrix H (row-major, overwritten):
// eigenvalues in w (ascending), eigenvectors as the columns of V.
void jacobi_hermitian(std::vector<cd>& H, int n, std::vector<double>& w, std::vector<cd>& V) {
  V.assign((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; i++) V[(size_t)i * n + i] = 1.0;
  auto at = [&](int i, int j) -> cd& { return H[(size_t)i * n + j]; };
  double total = 0;
  for (const cd& z : H) total += std::norm(z);
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0;
    for (int i = 0; i < n; i++)
      for (int j = i + 1; j < n; j++) off += std::norm(at(i, j));
    if (off <= 1e-30 * total || off == 0) break;
    for (int p = 0; p < n; p++)
      for (int q = p + 1; q < n; q++) {
        const cd g = at(p, q);
        const double r = std::abs(g);
        if (r <= 1e-300) continue;
        const cd ph = g / r;  // e^{i phi}
        const double a = at(p, p).real(), d = at(q, q).real();
        const double th = (d - a) / (2 * r);
        const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1));
        const double cs = 1 / sqrt(t * t + 1), sn = t * cs;
        // U = diag(1, conj(ph)) R, R = [[c, s], [-s, c]] in the (p, q) plane
        const cd Upp = cs, Upq = sn, Uqp = -sn * std::conj(ph), Uqq = cs * std::conj(ph);
        for (int k = 0; k < n; k++) {  // H <- H U
          const cd hp = at(k, p), hq = at(k, q);
          at(k, p) = hp * Upp + hq * Uqp;
          at(k, q) = hp * Upq + hq * Uqq;
        }
        for (int k = 0; k < n; k++) {  // H <- U^dag H
          const cd hp = at(p, k), hq = at(q, k);
          at(p, k) = std::conj(Upp) * hp + std::conj(Uqp) * hq;
          at(q, k) = std::conj(Upq) * hp + std::conj(Uqq) * hq;
        }
        for (int k = 0; k < n; k++) {  // V <- V U
          const cd vp = V[(size_t)k * n + p], vq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = vp * Upp + vq * Uqp;
          V[(size_t)k * n + q] = vp * Upq + vq * Uqq;
        }
        at(p, q) = 0;
        at(q, p) = 0;
      }
  }
  // sort ascending
  std::vector<int> idx(n);
  for (int i = 0; i < n; i++) idx[i] = i;
  for (int i = 1; i < n; i++)
    for (int j = i; j > 0 && at(idx[j], idx[j]).real() < at(idx[j - 1], idx[j - 1]).real(); j--) std::swap(idx[j], idx[j - 1]);
  std::vector<cd> V2((size_t)n * n);
  w.resize(n);
  for (int j = 0; j < n; j++) {
    w[j] = at(idx[j], idx[j]).real();
    for (int k = 0; k < n; k++) V2[(size_t)k * n + j] = V[(size_t)k * n + idx[j]];
  }
  V.swap(V2);
}

// A^2 v -> out via tmp (two stencil applies, FP32 CUDA cores).
int apply_aa(dwf_coarse* C, float2* out, const float2* v, float2* tmp, cudaStream_t st) {
  int rc = coarse_apply_dev(C, tmp, v, 1, st);
  if (rc) return rc;
  return coarse_apply_dev(C, out, tmp, 1, st);
}

// host scalars via the context's device scalar bank
int norm2_host(dwf_ctx* c, const void* v, int64_t n, double* out, cudaStream_t st) {
  int rc = norm2_dev(c, v, n, DWF_F32, S_TMP3, st);
  if (rc) return rc;
  rc = read_scalars(c, S_TMP3, 1, st);
  if (rc) return rc;
  *out = c->hscal[S_TMP3];
  return DWF_OK;
}

}  // namespace

void coarse_defl_free(dwf_coarse* C) {
  if (C->defl_V) cudaFree(C->defl_V);
  if (C->defl_thinv) cudaFree(C->defl_thinv);
  if (C->defl_c) cudaFree(C->defl_c);
  if (C->defl_tmp) cudaFree(C->defl_tmp);
  C->defl_V = nullptr;
  C->defl_thinv = nullptr;
  C->defl_c = nullptr;
  C->defl_tmp = nullptr;
  C->defl_nev = 0;
}

int coarse_defl_guess(dwf_coarse* C, const float2* r, cudaStream_t st) {
  dwf_ctx* c = C->ctx;
  const long long n = (long long)C->g.nc * C->nb;
  int rc = coarse_apply_dev(C, C->defl_tmp, r, 1, st);  // b = A r
  if (rc) return rc;
  c->launches += 2;
  k_multidot<<<C->defl_nev, DT, 0, st>>>(C->defl_V, n, C->defl_tmp, n, C->defl_c, C->defl_thinv);
  k_multicomb<<<comb_grid(n), DT, 0, st>>>(C->defl_tmp + n, C->defl_V, n, C->defl_nev, n, C->defl_c, 0.f, 1.0);
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

extern "C" int coarse_deflate(dwf_coarse* C, const void* v0, int nev, int nk, int order, double lam_lo,
                              double lam_max, double* theta, void* stream) {
  if (!C) return DWF_EINVAL;
  dwf_ctx* c = C->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  if (nev == 0) {  // drop the deflation space
    DWF_CUDA(c, cudaStreamSynchronize(st));
    coarse_defl_free(C);
    return DWF_OK;
  }
  if (!v0 || nev < 1 || nk < nev || nk > 1024 || order < 2 || (order & 1) || !(lam_lo > 0) ||
      !(lam_max <= 0 || lam_max > lam_lo))
    return dwf_fail(c, DWF_EINVAL, "coarse_deflate: bad arguments (need 1 <= nev <= nk <= 1024, even order >= 2, "
                                   "lam_lo > 0, lam_max <= 0 or > lam_lo)");
  const long long n = (long long)C->g.nc * C->nb;
  if (nk > n) return dwf_fail(c, DWF_EINVAL, "coarse_deflate: nk exceeds the coarse dimension");
  std::vector<void*> owned;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    owned.push_back(p);
    return p;
  };
  auto release = [&]() {
    for (void* p : owned) cudaFree(p);
    owned.clear();
  };
  float2* Q = (float2*)alloc((size_t)(nk + 1) * n * sizeof(float2));  // Lanczos basis
  float2* w = (float2*)alloc((size_t)n * sizeof(float2));
  float2* tp = (float2*)alloc((size_t)n * sizeof(float2));
  float2* tc = (float2*)alloc((size_t)n * sizeof(float2));
  float2* ax = (float2*)alloc((size_t)n * sizeof(float2));
  float2* tmp = (float2*)alloc((size_t)n * sizeof(float2));
  double2* cdev = (double2*)alloc((size_t)(nk + 1) * sizeof(double2));
  if (!Q || !w || !tp || !tc || !ax || !tmp || !cdev) {
    release();
    return dwf_fail(c, DWF_ENOMEM, "coarse_deflate workspace");
  }
  int rc = DWF_OK;
#define DEFL_TRY(call)  \
  do {                  \
    rc = (call);        \
    if (rc) {           \
      release();        \
      return rc;        \
    }                   \
  } while (0)
  // lambda_max of A^2 by the power method when not given (30 steps, +10 %)
  if (!(lam_max > 0)) {
    double nn = 0;
    DEFL_TRY(blas_copy(c, tp, DWF_F32, v0, DWF_F32, n, st));
    DEFL_TRY(norm2_host(c, tp, n, &nn, st));
    if (!(nn > 0)) {
      release();
      return dwf_fail(c, DWF_EINVAL, "coarse_deflate: zero start vector");
    }
    DEFL_TRY(blas_axpby(c, 1.0 / sqrt(nn), tp, DWF_F32, 0.0, tp, DWF_F32, n, st));
    double lam = 0;
    for (int k = 0; k < 30; k++) {
      DEFL_TRY(apply_aa(C, ax, tp, tmp, st));
      DEFL_TRY(norm2_host(c, ax, n, &nn, st));
      lam = sqrt(nn);  // |A^2 v| for unit v approaches the largest eigenvalue
      DEFL_TRY(blas_axpby(c, 1.0 / lam, ax, DWF_F32, 0.0, tp, DWF_F32, n, st));
    }
    lam_max = 1.1 * lam;
    if (!(lam_max > lam_lo)) {
      release();
      return dwf_fail(c, DWF_EINVAL, "coarse_deflate: lam_lo above the spectrum of A^2");
    }
  }
  const double ya = 2.0 / (lam_max - lam_lo), yb = -(lam_max + lam_lo) / (lam_max - lam_lo);
  // B v = T_order(y(A^2)) v into out (three-term recurrence)
  auto apply_B = [&](float2* out, const float2* v) -> int {
    int r = blas_copy(c, tp, DWF_F32, v, DWF_F32, n, st);
    if (r) return r;
    r = apply_aa(C, ax, tp, tmp, st);
    if (r) return r;
    r = blas_axpbypcz(c, ya, ax, yb, tp, 0.0, tc, n, DWF_F32, st);  // T_1
    if (r) return r;
    float2 *a = tp, *b = tc;
    for (int k = 2; k <= order; k++) {
      r = apply_aa(C, ax, b, tmp, st);
      if (r) return r;
      r = blas_cheb_step(c, a, ax, b, 2 * ya, 2 * yb, nullptr, 0.0, n, DWF_F32, st);  // a <- T_k
      if (r) return r;
      float2* t = a;
      a = b;
      b = t;
    }
    return blas_copy(c, out, DWF_F32, b, DWF_F32, n, st);
  };
  // Lanczos with full reorthogonalisation (classical Gram-Schmidt, twice)
  double nn = 0;
  DEFL_TRY(norm2_host(c, v0, n, &nn, st));
  if (!(nn > 0) || !isfinite(nn)) {
    release();
    return dwf_fail(c, DWF_EINVAL, "coarse_deflate: zero start vector");
  }
  DEFL_TRY(blas_axpby(c, 1.0 / sqrt(nn), v0, DWF_F32, 0.0, Q, DWF_F32, n, st));
  std::vector<double> alpha, beta;
  int k_steps = 0;
  for (int j = 0; j < nk; j++) {
    float2* qj = Q + (size_t)j * n;
    DEFL_TRY(apply_B(w, qj));
    int np = 0;
    DEFL_TRY(blas_cdot_partials(c, qj, w, n, DWF_F32, st, &np));
    DEFL_TRY(blas_finalize(c, np, 2, S_TMP0, st));
    DEFL_TRY(read_scalars(c, S_TMP0, 2, st));
    const double aj = c->hscal[S_TMP0];
    alpha.push_back(aj);
    DEFL_TRY(blas_axpby(c, -aj, qj, DWF_F32, 1.0, w, DWF_F32, n, st));
    if (j > 0) DEFL_TRY(blas_axpby(c, -beta[j - 1], Q + (size_t)(j - 1) * n, DWF_F32, 1.0, w, DWF_F32, n, st));
    for (int pass = 0; pass < 2; pass++) {
      c->launches += 2;
      k_multidot<<<j + 1, DT, 0, st>>>(Q, n, w, n, cdev, nullptr);
      k_multicomb<<<comb_grid(n), DT, 0, st>>>(w, Q, n, j + 1, n, cdev, 1.f, -1.0);
    }
    DWF_CUDA(c, cudaGetLastError());
    k_steps = j + 1;
    DEFL_TRY(norm2_host(c, w, n, &nn, st));
    const double bj = sqrt(nn);
    if (!isfinite(bj)) {
      release();
      return dwf_fail(c, DWF_ENAN, "coarse_deflate: Lanczos breakdown");
    }
    if (j == nk - 1 || bj < 1e-14) break;
    beta.push_back(bj);
    DEFL_TRY(blas_axpby(c, 1.0 / bj, w, DWF_F32, 0.0, Q + (size_t)(j + 1) * n, DWF_F32, n, st));
  }
  if (k_steps < nev) {
    release();
    return dwf_fail(c, DWF_ERANGE, "coarse_deflate: the Krylov space closed before nev vectors");
  }
  // eigenpairs of the tridiagonal matrix; B's nev largest -> W = Q S[:, top]
  const int k = k_steps;
  std::vector<cd> T((size_t)k * k, cd(0, 0)), S;
  for (int i = 0; i < k; i++) {
    T[(size_t)i * k + i] = alpha[i];
    if (i + 1 < k) T[(size_t)i * k + i + 1] = T[(size_t)(i + 1) * k + i] = beta[i];
  }
  std::vector<double> mu;
  jacobi_hermitian(T, k, mu, S);
  float2* W = (float2*)alloc((size_t)nev * n * sizeof(float2));
  float2* AW = (float2*)alloc((size_t)nev * n * sizeof(float2));
  if (!W || !AW) {
    release();
    return dwf_fail(c, DWF_ENOMEM, "coarse_deflate workspace");
  }
  std::vector<double2> col(k);
  for (int t = 0; t < nev; t++) {
    const int src = k - 1 - t;  // largest first
    for (int i = 0; i < k; i++) col[i] = make_double2(S[(size_t)i * k + src].real(), S[(size_t)i * k + src].imag());
    DWF_CUDA(c, cudaMemcpyAsync(cdev, col.data(), k * sizeof(double2), cudaMemcpyHostToDevice, st));
    c->launches++;
    k_multicomb<<<comb_grid(n), DT, 0, st>>>(W + (size_t)t * n, Q, n, k, n, cdev, 0.f, 1.0);
    DWF_CUDA(c, cudaStreamSynchronize(st));  // col is reused
  }
  // Rayleigh-Ritz with A^2 on span(W): H_st = <w_s, A^2 w_t>
  for (int t = 0; t < nev; t++) DEFL_TRY(apply_aa(C, AW + (size_t)t * n, W + (size_t)t * n, tmp, st));
  std::vector<cd> H((size_t)nev * nev);
  std::vector<double2> hcol(nev);
  for (int t = 0; t < nev; t++) {
    c->launches++;
    k_multidot<<<nev, DT, 0, st>>>(W, n, AW + (size_t)t * n, n, cdev, nullptr);
    DWF_CUDA(c, cudaMemcpyAsync(hcol.data(), cdev, nev * sizeof(double2), cudaMemcpyDeviceToHost, st));
    DWF_CUDA(c, cudaStreamSynchronize(st));
    for (int s2 = 0; s2 < nev; s2++) H[(size_t)s2 * nev + t] = cd(hcol[s2].x, hcol[s2].y);
  }
  for (int s2 = 0; s2 < nev; s2++)  // symmetrise (rounding)
    for (int t = s2; t < nev; t++) {
      const cd a = 0.5 * (H[(size_t)s2 * nev + t] + std::conj(H[(size_t)t * nev + s2]));
      H[(size_t)s2 * nev + t] = a;
      H[(size_t)t * nev + s2] = std::conj(a);
    }
  std::vector<double> th;
  std::vector<cd> Cm;
  jacobi_hermitian(H, nev, th, Cm);
  for (int t = 0; t < nev; t++)
    if (!(th[t] > 0)) {
      release();
      return dwf_fail(c, DWF_ERANGE, "coarse_deflate: non-positive Ritz value of A^2");
    }
  // keep V = W C and 1/theta with the operator
  coarse_defl_free(C);
  void *V = nullptr, *ti = nullptr, *cc = nullptr, *tt = nullptr;
  if (cudaMalloc(&V, (size_t)nev * n * sizeof(float2)) != cudaSuccess || cudaMalloc(&ti, nev * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&cc, nev * sizeof(double2)) != cudaSuccess || cudaMalloc(&tt, 2 * (size_t)n * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    if (V) cudaFree(V);
    if (ti) cudaFree(ti);
    if (cc) cudaFree(cc);
    if (tt) cudaFree(tt);
    release();
    return dwf_fail(c, DWF_ENOMEM, "coarse deflation space");
  }
  C->defl_V = (float2*)V;
  C->defl_thinv = (double*)ti;
  C->defl_c = (double2*)cc;
  C->defl_tmp = (float2*)tt;
  std::vector<double> thinv(nev);
  for (int t = 0; t < nev; t++) {
    for (int s2 = 0; s2 < nev; s2++) hcol[s2] = make_double2(Cm[(size_t)s2 * nev + t].real(), Cm[(size_t)s2 * nev + t].imag());
    DWF_CUDA(c, cudaMemcpyAsync(cdev, hcol.data(), nev * sizeof(double2), cudaMemcpyHostToDevice, st));
    c->launches++;
    k_multicomb<<<comb_grid(n), DT, 0, st>>>(C->defl_V + (size_t)t * n, W, n, nev, n, cdev, 0.f, 1.0);
    DWF_CUDA(c, cudaStreamSynchronize(st));
    thinv[t] = 1.0 / th[t];
    if (theta) theta[t] = th[t];
  }
  DWF_CUDA(c, cudaMemcpy(C->defl_thinv, thinv.data(), nev * sizeof(double), cudaMemcpyHostToDevice));
  C->defl_nev = nev;
  release();
#undef DEFL_TRY
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

extern "C" int coarse_export_deflation(const dwf_coarse* C, void* V, double* theta_inv, int* nev) {
  if (!C) return DWF_EINVAL;
  if (nev) *nev = C->defl_nev;
  const long long n = (long long)C->g.nc * C->nb;
  if (V && C->defl_nev > 0 &&
      cudaMemcpy(V, C->defl_V, (size_t)C->defl_nev * n * sizeof(float2), cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return DWF_ECUDA;
  }
  if (theta_inv && C->defl_nev > 0 &&
      cudaMemcpy(theta_inv, C->defl_thinv, C->defl_nev * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return DWF_ECUDA;
  }
  return DWF_OK;
}
