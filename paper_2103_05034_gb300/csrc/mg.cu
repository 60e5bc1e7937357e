// HDCR multigrid (arXiv:2103.05034, Secs. 3.1-3.4, Table 1): Chebyshev
// filters, chirality projection, block Cholesky-QR orthonormalisation, the
// 9-point little Dirac operator of H_DW, coarse CG on A^2, the Chebyshev
// smoother, the V(1,1) preconditioner and the flexible GCR outer solver.
#include <math.h>
#include <string.h>

#include <chrono>
#include <new>
#include <vector>

#include "coarse_internal.cuh"

struct dwf_mg {
  dwf_ctx* ctx;
  dwf_mg_params p;
  BlockGeom g;
  float2* basis;  // nb full FP32 fields
  dwf_coarse* coarse;
  dwf_hybrid* hyb;  // the levels of the hybrid three-level multigrid, or null
  double lambda_max_used;
  double setup_seconds, coarse_op_seconds;
};

namespace {

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double sec() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

int64_t full_elems(const dwf_ctx* c) { return 2 * c->g.Vh * 12 * c->g.Ls; }

int make_geom(dwf_ctx* c, const int block[4], BlockGeom* g) {
  int b4 = 1, nc = 1;
  for (int m = 0; m < 4; m++) {
    if (block[m] < 1 || c->g.L[m] % block[m]) return dwf_fail(c, DWF_EINVAL, "block does not tile the lattice");
    g->L[m] = c->g.L[m];
    g->b[m] = block[m];
    g->Lc[m] = c->g.L[m] / block[m];
    b4 *= block[m];
    nc *= g->Lc[m];
  }
  g->Lxh = c->g.Lxh;
  g->Vh = (int)c->g.Vh;
  g->Ls = c->g.Ls;
  g->b4 = b4;
  g->nc = nc;
  return DWF_OK;
}

// Workspace slots used here (the solver slots of api.cu end at 15).
enum { MW_T0 = 16, MW_T1, MW_T2, MW_T3, MW_T4, MW_T5, MW_T6, MW_T7, MW_T8, MW_T9, MW_T10, MW_T11 };

void* ws(dwf_ctx* c, int slot, size_t bytes) { return dwf_workspace(c, slot, bytes); }

// D^dag D on nrhs full fields via tmp; with cf the result feeds cf's
// Chebyshev step instead of out (fused into the last hopping launches).
int mdagm(dwf_ctx* c, void* out, const void* in, void* tmp, double mf, int prec, int nrhs, cudaStream_t st,
          const ChebFuse* cf = nullptr) {
  std::vector<double> m(nrhs, mf);
  int rc = ddw_apply(c, tmp, in, m.data(), 0, 0, prec, nrhs, st);
  if (rc) return rc;
  return ddw_apply(c, out, tmp, m.data(), 1, 0, prec, nrhs, st, cf);
}

// H_DW^2 on nrhs full fields via tmp (cf as for mdagm).
int hsq(dwf_ctx* c, void* out, const void* in, void* tmp, double mf, int prec, int nrhs, cudaStream_t st,
        const ChebFuse* cf = nullptr) {
  std::vector<double> m(nrhs, mf);
  int rc = ddw_apply(c, tmp, in, m.data(), 0, 1, prec, nrhs, st);
  if (rc) return rc;
  return ddw_apply(c, out, tmp, m.data(), 0, 1, prec, nrhs, st, cf);
}

int check_finite(dwf_ctx* c, const void* v, int64_t n, int prec, cudaStream_t st, double* norm2) {
  int rc = norm2_dev(c, v, n, prec, S_TMP3, st);
  if (rc) return rc;
  rc = read_scalars(c, S_TMP3, 1, st);
  if (rc) return rc;
  if (norm2) *norm2 = c->hscal[S_TMP3];
  if (!isfinite(c->hscal[S_TMP3])) return dwf_fail(c, DWF_ERANGE, "Chebyshev filter overflow: spectrum outside [lo, hi]");
  return DWF_OK;
}

// T_order(x(A)) in -> out on nrhs full fields, x(A) = 2(A-lo)/(hi-lo) - 1, A = D^dag D.
// With rescale, the pair (T_k, T_{k-1}) is divided by a common factor whenever
// it grows past 1e15 (directions are kept, magnitudes are not).
int filter_core(dwf_ctx* c, void* out, const void* in, int nrhs, double lo, double hi, int order, double mf,
                int prec, bool rescale, cudaStream_t st, void** tprev_out = nullptr, void** tcur_out = nullptr) {
  const int64_t n = full_elems(c) * nrhs;
  const size_t bytes = n * dwf_complex_bytes(prec);
  void* tp = ws(c, MW_T0, bytes);
  void* tc = ws(c, MW_T1, bytes);
  void* ax = ws(c, MW_T2, bytes);
  void* tmp = ws(c, MW_T3, bytes);
  if (!tp || !tc || !ax || !tmp) return dwf_fail(c, DWF_ENOMEM, "filter workspace");
  const double a = 2.0 / (hi - lo), b = -(hi + lo) / (hi - lo);
  int rc = blas_copy(c, tp, prec, in, prec, n, st);
  if (rc) return rc;
  if (order == 0) return blas_copy(c, out, prec, tp, prec, n, st);
  rc = mdagm(c, ax, tp, tmp, mf, prec, nrhs, st);
  if (rc) return rc;
  rc = blas_axpbypcz(c, a, ax, b, tp, 0.0, tc, n, prec, st);  // T1 = x(A) T0
  if (rc) return rc;
  for (int k = 2; k <= order; k++) {
    // tp <- T_k = 2 x(A) T_{k-1} - T_{k-2}, the step fused into the last hops
    const ChebFuse cf = {tc, tp, nullptr, 2 * a, 2 * b, 0.0};
    rc = mdagm(c, ax, tc, tmp, mf, prec, nrhs, st, &cf);
    if (rc) return rc;
    void* t = tp;
    tp = tc;
    tc = t;
    if (rescale && k % 16 == 0) {
      double nn = 0;
      rc = check_finite(c, tc, n, prec, st, &nn);
      if (rc) return rc;
      if (nn > 1e30) {
        const double f = 1.0 / sqrt(nn);
        rc = blas_axpby(c, f, tc, prec, 0.0, tc, prec, n, st);
        if (rc) return rc;
        rc = blas_axpby(c, f, tp, prec, 0.0, tp, prec, n, st);
        if (rc) return rc;
      }
    }
  }
  if (tprev_out) {
    *tprev_out = tp;
    *tcur_out = tc;
  }
  if (out) return blas_copy(c, out, prec, tc, prec, n, st);
  return DWF_OK;
}

// Normalise each of nrhs fields of n complex numbers to unit norm (host loop).
int normalise_fields(dwf_ctx* c, void* v, int nrhs, int64_t n, int prec, cudaStream_t st) {
  const size_t cb = dwf_complex_bytes(prec);
  for (int r = 0; r < nrhs; r++) {
    char* p = (char*)v + r * n * cb;
    double nn = 0;
    int rc = check_finite(c, p, n, prec, st, &nn);
    if (rc) return rc;
    if (!(nn > 0)) return dwf_fail(c, DWF_ERANGE, "filtered vector vanished");
    rc = blas_axpby(c, 1.0 / sqrt(nn), p, prec, 0.0, p, prec, n, st);
    if (rc) return rc;
  }
  return DWF_OK;
}

template <int P>
void launch_chiral(void* out, const void* in, long long n, int Ls, float sign, cudaStream_t st) {
  dwfmg::k_chiral_project<P><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      (typename Prec<P>::S*)out, (const typename Prec<P>::S*)in, n, Ls, sign);
}

int chiral(dwf_ctx* c, void* out, const void* in, int sign, int prec, int nrhs, cudaStream_t st) {
  const long long n = full_elems(c) * nrhs;
  c->launches++;
  switch (prec) {
    case DWF_F64:
      launch_chiral<DWF_F64>(out, in, n, c->g.Ls, (float)sign, st);
      break;
    case DWF_F32:
      launch_chiral<DWF_F32>(out, in, n, c->g.Ls, (float)sign, st);
      break;
    default:
      return dwf_fail(c, DWF_EINVAL, "bad precision");
  }
  return DWF_OK;
}

// out[xc][j][k] = <X_j, Y_k>_block (face-restricted for d > 0), FP64 results.
int block_inner(dwf_ctx* c, const BlockGeom& g, const void* X, int nx, const void* Y, int ny, int prec,
                double2* out, long long out_bstride, int out_ld, int d, int accumulate, cudaStream_t st) {
  const long long fs = full_elems(c);
  c->launches++;
  if (ny == 1 && d == 0 && !accumulate && nx <= 64 && (prec == DWF_F32 || prec == DWF_F64)) {
    // restriction of one field: nx dot products per block in one pass
#define DWF_RESTRICT(PV, NXV)                                                                                  \
  dwfmg::k_block_restrict<PV, NXV><<<g.nc, 256, 0, st>>>((const typename Prec<PV>::S*)X, fs, nx,               \
                                                         (const typename Prec<PV>::S*)Y, out, out_bstride, out_ld, g)
    if (prec == DWF_F32) {
      if (nx <= 8) DWF_RESTRICT(DWF_F32, 8);
      else if (nx <= 32) DWF_RESTRICT(DWF_F32, 32);
      else DWF_RESTRICT(DWF_F32, 64);
    } else {
      if (nx <= 8) DWF_RESTRICT(DWF_F64, 8);
      else if (nx <= 32) DWF_RESTRICT(DWF_F64, 32);
      else DWF_RESTRICT(DWF_F64, 64);
    }
#undef DWF_RESTRICT
    return DWF_OK;
  }
  dim3 grid(g.nc, (nx + 31) / 32, (ny + 31) / 32);
  switch (prec) {
    case DWF_F64:
      dwfmg::k_block_inner<DWF_F64><<<grid, 256, 0, st>>>((const double2*)X, fs, nx, (const double2*)Y, fs, ny,
                                                          out, out_bstride, out_ld, g, d, accumulate);
      break;
    case DWF_F32:
      dwfmg::k_block_inner<DWF_F32><<<grid, 256, 0, st>>>((const float2*)X, fs, nx, (const float2*)Y, fs, ny,
                                                          out, out_bstride, out_ld, g, d, accumulate);
      break;
    default:
      return dwf_fail(c, DWF_EINVAL, "bad precision");
  }
  return DWF_OK;
}

// Y_k = sum_j X_j M[xc][j][k] per block (Y += when accumulate).
int block_combine(dwf_ctx* c, const BlockGeom& g, void* Y, int ny, int py, const void* X, int nx, int px,
                  const double2* M, long long m_bstride, int m_ld, int accumulate, cudaStream_t st) {
  if (nx * ny > 1024) return dwf_fail(c, DWF_EINVAL, "block combine too wide");
  const long long fs = full_elems(c);
  c->launches++;
  if (px == DWF_F64 && py == DWF_F64)
    dwfmg::k_block_combine<DWF_F64, DWF_F64><<<g.nc, 256, 0, st>>>((double2*)Y, fs, ny, (const double2*)X, fs,
                                                                   nx, M, m_bstride, m_ld, g, accumulate);
  else if (px == DWF_F32 && py == DWF_F32)
    dwfmg::k_block_combine<DWF_F32, DWF_F32><<<g.nc, 256, 0, st>>>((float2*)Y, fs, ny, (const float2*)X, fs,
                                                                   nx, M, m_bstride, m_ld, g, accumulate);
  else
    return dwf_fail(c, DWF_EINVAL, "bad precision pair");
  return DWF_OK;
}

}  // namespace

void dwf_ws_release(dwf_ctx* c, int slot) {
  if (slot < 0 || slot >= DWF_NWS || !c->ws[slot]) return;
  cudaFree(c->ws[slot]);
  c->ws[slot] = nullptr;
  c->ws_bytes[slot] = 0;
}

namespace {

// Block Cholesky-QR on nb FP32 full fields in place (FP64 Gram sums and
// factorisation, FP32 update arithmetic): the basis orthonormalisation of the
// multigrid setup without an FP64 copy of the basis.  Three passes, the first
// with the Gram matrix shifted by 1e-5 of its largest diagonal entry (shifted
// Cholesky-QR: the filtered vectors can be dependent to FP32 precision on a
// block, and a plain Cholesky factorisation of their Gram matrix then fails);
// the first pass brings the condition number to about 300, the next two
// orthonormalise.  Every pass multiplies by an upper-triangular matrix with a
// positive diagonal, so the result is the Q of the QR factorisation (the same
// vectors as Gram-Schmidt in exact arithmetic).
int ortho_inplace_f32(dwf_ctx* c, const BlockGeom& g, float2* basis, int nb, int nplus, cudaStream_t st) {
  const int64_t n = full_elems(c);
  const size_t gbytes = (size_t)g.nc * nb * nb * sizeof(double2);
  double2* Gm = (double2*)ws(c, MW_T8, gbytes);
  double2* Ri = (double2*)ws(c, MW_T9, gbytes);
  int* fail = (int*)ws(c, MW_T11, sizeof(int) * 4);
  if (!Gm || !Ri || !fail) return dwf_fail(c, DWF_ENOMEM, "orthonormalisation workspace");
  for (int pass = 0; pass < 3; pass++) {
    int rc = block_inner(c, g, basis, nb, basis, nb, DWF_F32, Gm, (long long)nb * nb, nb, 0, 0, st);
    if (rc) return rc;
    DWF_CUDA(c, cudaMemsetAsync(Ri, 0, gbytes, st));
    DWF_CUDA(c, cudaMemsetAsync(fail, 0, sizeof(int), st));
    c->launches++;
    dwfmg::k_block_cholinv<<<dim3(g.nc, 2), 32, 0, st>>>(Gm, Ri, nb, nplus, fail, pass == 0 ? 1e-5 : 0.0);
    for (int grp = 0; grp < 2; grp++) {
      const int g0 = grp ? nplus : 0, ng = grp ? nb - nplus : nplus;
      if (ng <= 0) continue;
      c->launches++;
      dwfmg::k_block_update_inplace<<<g.nc, 256, 0, st>>>(basis + (size_t)g0 * n, n, ng, g0, nb, Ri, g);
    }
    int hfail = 0;
    DWF_CUDA(c, cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CUDA(c, cudaStreamSynchronize(st));
    if (hfail) return dwf_fail(c, DWF_ERANGE, "basis vectors linearly dependent on a block");
  }
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

}  // namespace

int coarse_ws(dwf_coarse* C, int slot, size_t bytes, void** out) {
  if (C->ws_bytes[slot] < bytes || !C->ws[slot]) {
    if (C->ws[slot]) cudaFree(C->ws[slot]);
    C->ws[slot] = nullptr;
    C->ws_bytes[slot] = 0;
    if (cudaMalloc(&C->ws[slot], bytes) != cudaSuccess) {
      cudaGetLastError();
      return dwf_fail(C->ctx, DWF_ENOMEM, "coarse workspace");
    }
    C->ws_bytes[slot] = bytes;
  }
  *out = C->ws[slot];
  return DWF_OK;
}

int coarse_apply_dev(dwf_coarse* C, float2* out, const float2* in, int nrhs, cudaStream_t st) {
  const long long n = (long long)C->g.nc * C->nb * nrhs;
  C->ctx->launches++;
  // fewer than 32 right-hand sides: a warp of the one-output kernel spans
  // several operator rows, so four outputs per thread issue fewer loads; from
  // 32 on, a warp shares one operator element and reads 256 contiguous bytes
  if ((nrhs & 3) == 0 && nrhs < 32 && (((uintptr_t)in | (uintptr_t)out) & 15) == 0) {
    const unsigned b4 = (unsigned)((n / 4 + 255) / 256);
#define DWF_CA4(NBV)                                                                                            \
  dwfmg::k_coarse_apply4<NBV><<<b4, 256, 0, st>>>(out, in, C->A32, C->g.Lc[0], C->g.Lc[1], C->g.Lc[2], C->g.Lc[3], \
                                                  C->nb, nrhs)
    switch (C->nb) {
      case 16: DWF_CA4(16); break;
      case 24: DWF_CA4(24); break;
      case 32: DWF_CA4(32); break;
      default: DWF_CA4(0); break;
    }
#undef DWF_CA4
    return DWF_OK;
  }
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (C->nb == 32)
    dwfmg::k_coarse_apply<32><<<blocks, 256, 0, st>>>(out, in, C->A32, C->g.Lc[0], C->g.Lc[1], C->g.Lc[2],
                                                      C->g.Lc[3], C->nb, nrhs);
  else if (C->nb == 24)  // the hybrid multigrid's 4D basis (Algorithm F)
    dwfmg::k_coarse_apply<24><<<blocks, 256, 0, st>>>(out, in, C->A32, C->g.Lc[0], C->g.Lc[1], C->g.Lc[2],
                                                      C->g.Lc[3], C->nb, nrhs);
  else if (C->nb == 16)
    dwfmg::k_coarse_apply<16><<<blocks, 256, 0, st>>>(out, in, C->A32, C->g.Lc[0], C->g.Lc[1], C->g.Lc[2],
                                                      C->g.Lc[3], C->nb, nrhs);
  else
    dwfmg::k_coarse_apply<0><<<blocks, 256, 0, st>>>(out, in, C->A32, C->g.Lc[0], C->g.Lc[1], C->g.Lc[2],
                                                     C->g.Lc[3], C->nb, nrhs);
  return DWF_OK;
}

// CG on A^2 e = A r (one right-hand side, FP32 vectors), stopping when the
// normal-equation residual falls below tol times its initial value: one
// persistent cooperative launch (coarse_cg.cu).
int coarse_cg(dwf_coarse* C, float2* e, const float2* rc, double tol, int maxiter, int* iters, cudaStream_t st) {
  const int64_t n = (int64_t)C->g.nc * C->nb;
  const int part_cap = 3 * 4096;
  void *work, *part, *small;
  int rc2;
  if ((rc2 = coarse_ws(C, 0, 4 * n * sizeof(float2), &work)) || (rc2 = coarse_ws(C, 1, part_cap * sizeof(double), &part)) ||
      (rc2 = coarse_ws(C, 2, CG_SMALL_BYTES, &small)))
    return rc2;
  // with a deflation space the CG starts from its guess (coarse_deflate)
  const float2* x0 = nullptr;
  if (C->defl_nev > 0) {
    rc2 = coarse_defl_guess(C, rc, st);
    if (rc2) return rc2;
    x0 = C->defl_tmp + n;
  }
  return coarse_cg_persistent(C->ctx, e, rc, C->A32, C->g.Lc, C->g.nc, C->nb, tol, maxiter, (float2*)work,
                              (double*)part, part_cap, (int*)small, C->cg_acc, iters, st, x0);
}

// The red-black form of the operator, built once (synchronises when it is built).
int coarse_rb_ready(dwf_coarse* C, cudaStream_t st) {
  if (C->Arb) return DWF_OK;
  for (int m = 0; m < 4; m++)
    if (C->g.Lc[m] & 1) return dwf_fail(C->ctx, DWF_EINVAL, "red-black coarse solve needs even coarse extents");
  const size_t na = (size_t)C->g.nc * 9 * C->nb * C->nb;
  void* small;
  int rc = coarse_ws(C, 2, CG_SMALL_BYTES, &small);
  if (rc) return rc;
  if (cudaMalloc(&C->Arb, na * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    C->Arb = nullptr;
    return dwf_fail(C->ctx, DWF_ENOMEM, "red-black coarse operator");
  }
  rc = coarse_rb_prepare(C->ctx, C->A64, C->Arb, C->g.Lc, C->g.nc, C->nb, (int*)small, st);
  if (rc) {
    cudaFree(C->Arb);
    C->Arb = nullptr;
  }
  return rc;
}

// Red-black CG on S^2 (coarse_cg.cu): same contract as coarse_cg.
int coarse_rbcg(dwf_coarse* C, float2* e, const float2* rc, double tol, int maxiter, int* iters, cudaStream_t st) {
  int r = coarse_rb_ready(C, st);
  if (r) return r;
  const int64_t n = (int64_t)C->g.nc * C->nb;
  const int part_cap = 3 * 4096;
  void *work, *part, *small;
  if ((r = coarse_ws(C, 3, 7 * n * sizeof(float2), &work)) || (r = coarse_ws(C, 1, part_cap * sizeof(double), &part)) ||
      (r = coarse_ws(C, 2, CG_SMALL_BYTES, &small)))
    return r;
  return coarse_rbcg_persistent(C->ctx, e, rc, C->Arb, C->g.Lc, C->g.nc, C->nb, tol, maxiter, (float2*)work,
                                (double*)part, part_cap, (int*)small, C->cg_acc, iters, st);
}

// ====================================================================== ABI

extern "C" int cheby_filter(dwf_ctx* c, void* out, const void* in, int nrhs, double lo, double hi, int order,
                            double mf, int prec, void* stream) {
  if (!c || !out || !in) return DWF_EINVAL;
  if (nrhs < 1 || nrhs > DWF_MAX_RHS || order < 0 || !(hi > lo)) return dwf_fail(c, DWF_EINVAL, "bad filter arguments");
  if (prec != DWF_F64 && prec != DWF_F32) return dwf_fail(c, DWF_EINVAL, "bad precision");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = filter_core(c, out, in, nrhs, lo, hi, order, mf, prec, false, st);
  if (rc) return rc;
  rc = check_finite(c, out, full_elems(c) * nrhs, prec, st, nullptr);
  if (rc) return rc;
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

extern "C" int cheby_recursive_basis(dwf_ctx* c, void* phi, const void* eta, double lam_lo, double lam_max, int m,
                                     int delta, int nvec, double mf, int prec, void* stream) {
  if (!c || !phi || !eta) return DWF_EINVAL;
  if (nvec < 1 || m < 0 || delta < 1 || !(lam_max > lam_lo)) return dwf_fail(c, DWF_EINVAL, "bad filter arguments");
  if (prec != DWF_F64 && prec != DWF_F32) return dwf_fail(c, DWF_EINVAL, "bad precision");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = full_elems(c);
  const size_t cb = dwf_complex_bytes(prec);
  // pre-filter (Eq. 34) into phi_0, normalised
  int rc = filter_core(c, phi, eta, 1, lam_lo, lam_max, m, mf, prec, true, st);
  if (rc) return rc;
  rc = normalise_fields(c, phi, 1, n, prec, st);
  if (rc) return rc;
  // one recurrence of T_n(2A/lam_max - 1) phi_0 with snapshots at k*delta (Eqs. 35, 37)
  const size_t bytes = n * cb;
  void* tp = ws(c, MW_T4, bytes);
  void* tc = ws(c, MW_T5, bytes);
  void* ax = ws(c, MW_T6, bytes);
  void* tmp = ws(c, MW_T7, bytes);
  if (!tp || !tc || !ax || !tmp) return dwf_fail(c, DWF_ENOMEM, "filter workspace");
  const double a = 2.0 / lam_max, b = -1.0;
  rc = blas_copy(c, tp, prec, phi, prec, n, st);
  if (rc) return rc;
  int order = 0;
  for (int k = 1; k < nvec; k++) {
    while (order < k * delta) {
      if (order == 0) {
        rc = mdagm(c, ax, tp, tmp, mf, prec, 1, st);
        if (rc) return rc;
        rc = blas_axpbypcz(c, a, ax, b, tp, 0.0, tc, n, prec, st);
      } else {
        const ChebFuse cf = {tc, tp, nullptr, 2 * a, 2 * b, 0.0};
        rc = mdagm(c, ax, tc, tmp, mf, prec, 1, st, &cf);
        void* t = tp;
        tp = tc;
        tc = t;
      }
      if (rc) return rc;
      order++;
    }
    char* dst = (char*)phi + k * bytes;
    rc = blas_copy(c, dst, prec, tc, prec, n, st);
    if (rc) return rc;
    rc = normalise_fields(c, dst, 1, n, prec, st);
    if (rc) return rc;
  }
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

extern "C" int dwf_chiral_project(dwf_ctx* c, void* out, const void* in, int sign, int prec, int nrhs,
                                  void* stream) {
  if (!c || !out || !in || (sign != 1 && sign != -1)) return DWF_EINVAL;
  if (nrhs < 1) return dwf_fail(c, DWF_EINVAL, "nrhs");
  int rc = chiral(c, out, in, sign, prec, nrhs, (cudaStream_t)stream);
  if (rc) return rc;
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

extern "C" int block_orthonormalise(dwf_ctx* c, void* basis, int nb, int nplus, const int block[4], void* stream) {
  if (!c || !basis || !block) return DWF_EINVAL;
  if (nb < 1 || nplus < 0 || nplus > nb || nplus > 32 || nb - nplus > 32)
    return dwf_fail(c, DWF_EINVAL, "groups of at most 32 vectors");
  BlockGeom g;
  int rc = make_geom(c, block, &g);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = full_elems(c);
  const size_t gbytes = (size_t)g.nc * nb * nb * sizeof(double2);
  double2* G = (double2*)ws(c, MW_T8, gbytes);
  double2* Ri = (double2*)ws(c, MW_T9, gbytes);
  void* tmp = ws(c, MW_T10, (size_t)n * nb * 16);
  int* fail = (int*)ws(c, MW_T11, sizeof(int) * 4);
  if (!G || !Ri || !tmp || !fail) return dwf_fail(c, DWF_ENOMEM, "orthonormalisation workspace");
  for (int pass = 0; pass < 2; pass++) {  // Cholesky-QR, twice
    rc = block_inner(c, g, basis, nb, basis, nb, DWF_F64, G, (long long)nb * nb, nb, 0, 0, st);
    if (rc) return rc;
    DWF_CUDA(c, cudaMemsetAsync(Ri, 0, gbytes, st));
    DWF_CUDA(c, cudaMemsetAsync(fail, 0, sizeof(int), st));
    c->launches++;
    dwfmg::k_block_cholinv<<<dim3(g.nc, 2), 32, 0, st>>>(G, Ri, nb, nplus, fail);
    // R^-1 is block diagonal by chirality group: update each group separately
    for (int grp = 0; grp < 2; grp++) {
      const int g0 = grp ? nplus : 0, ng = grp ? nb - nplus : nplus;
      if (ng <= 0) continue;
      rc = block_combine(c, g, (double2*)tmp + (size_t)g0 * n, ng, DWF_F64, (const double2*)basis + (size_t)g0 * n,
                         ng, DWF_F64, Ri + (size_t)g0 * nb + g0, (long long)nb * nb, nb, 0, st);
      if (rc) return rc;
    }
    DWF_CUDA(c, cudaMemcpyAsync(basis, tmp, (size_t)n * nb * 16, cudaMemcpyDeviceToDevice, st));
    int hfail = 0;
    DWF_CUDA(c, cudaMemcpyAsync(&hfail, fail, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CUDA(c, cudaStreamSynchronize(st));
    if (hfail) return dwf_fail(c, DWF_ERANGE, "basis vectors linearly dependent on a block");
  }
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

// ---------------------------------------------------------------------- coarse operator
extern "C" int coarse_build(dwf_ctx* c, const void* basis, int nb, int nplus, const int block[4], double mf,
                            int prec, dwf_coarse** out, void* stream) {
  if (!c || !basis || !block || !out) return DWF_EINVAL;
  *out = nullptr;
  if (nb < 1 || nb > DWF_MAX_RHS || nplus < 0 || nplus > nb) return dwf_fail(c, DWF_EINVAL, "bad nbasis");
  if (prec != DWF_F64 && prec != DWF_F32) return dwf_fail(c, DWF_EINVAL, "bad precision");
  BlockGeom g;
  int rc = make_geom(c, block, &g);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  dwf_coarse* C = new (std::nothrow) dwf_coarse();
  if (!C) return DWF_ENOMEM;
  C->ctx = c;
  C->g = g;
  C->nb = nb;
  C->nplus = nplus;
  const size_t na = (size_t)g.nc * 9 * nb * nb;
  if (cudaMalloc(&C->A64, na * sizeof(double2)) != cudaSuccess || cudaMalloc(&C->A32, na * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    coarse_destroy(C);
    return dwf_fail(c, DWF_ENOMEM, "coarse operator");
  }
  // H_DW phi_k and its eight face terms for a group of basis vectors at a
  // time (workspace: two groups of full fields); the block inner products
  // with every basis vector fill those columns of A.  Each group re-reads the
  // whole basis once per direction, so the group is as wide as free device
  // memory allows (all nb vectors at small volumes, 8 at the largest).
  const int64_t n = full_elems(c);
  const size_t cbytes = dwf_complex_bytes(prec);
  int ngmax = nb < 8 ? nb : 8;
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess) {
      const size_t margin = (size_t)4 << 30;
      for (int cand = nb; cand > ngmax; cand = (cand + 1) / 2) {
        if (2 * (size_t)n * cand * cbytes + margin < fr) {
          ngmax = cand;
          break;
        }
      }
    } else {
      cudaGetLastError();
    }
  }
  const size_t fb = (size_t)n * ngmax * cbytes;
  void* H = ws(c, MW_T8, fb);
  void* W = ws(c, MW_T9, fb);
  if (!H || !W) {
    coarse_destroy(C);
    return dwf_fail(c, DWF_ENOMEM, "coarse build workspace");
  }
  const long long bstride = 9LL * nb * nb;
  for (int k0 = 0; k0 < nb && rc == DWF_OK; k0 += ngmax) {
    const int ng = nb - k0 < ngmax ? nb - k0 : ngmax;
    const void* bk = (const char*)basis + (size_t)k0 * n * cbytes;
    std::vector<double> m(ng, mf);
    rc = ddw_apply(c, H, bk, m.data(), 0, 1, prec, ng, st);
    for (int d = 1; d <= 8 && rc == DWF_OK; d++) {
      const unsigned nblk = (unsigned)((2LL * g.Vh * g.Ls + 127) / 128);
      dim3 grid(nblk, ng);
      c->launches++;
#define DWF_FACE(PV, LSV)                                                                                  \
  dwfmg::k_face_hop<PV, LSV><<<grid, 128, 0, st>>>((typename Prec<PV>::S*)W,                                \
                                                    (const typename Prec<PV>::S*)bk, n,                    \
                                                    (const typename Prec<PV>::LS*)(PV == DWF_F64 ? (void*)c->links64[0] : (void*)c->links32[0]), \
                                                    (const typename Prec<PV>::LS*)(PV == DWF_F64 ? (void*)c->links64[1] : (void*)c->links32[1]), g, d)
      if (prec == DWF_F64) {
        switch (g.Ls) {
          case 4: DWF_FACE(DWF_F64, 4); break;
          case 8: DWF_FACE(DWF_F64, 8); break;
          case 16: DWF_FACE(DWF_F64, 16); break;
          default: DWF_FACE(DWF_F64, 24); break;
        }
      } else {
        switch (g.Ls) {
          case 4: DWF_FACE(DWF_F32, 4); break;
          case 8: DWF_FACE(DWF_F32, 8); break;
          case 16: DWF_FACE(DWF_F32, 16); break;
          default: DWF_FACE(DWF_F32, 24); break;
        }
      }
#undef DWF_FACE
      rc = block_inner(c, g, basis, nb, W, ng, prec, C->A64 + (size_t)d * nb * nb + k0, bstride, nb, d, 0, st);
      if (rc) break;
      rc = blas_axpby(c, -1.0, W, prec, 1.0, H, prec, n * ng, st);
    }
    if (rc == DWF_OK) rc = block_inner(c, g, basis, nb, H, ng, prec, C->A64 + k0, bstride, nb, 0, 0, st);
  }
  if (rc == DWF_OK) rc = blas_copy(c, C->A32, DWF_F32, C->A64, DWF_F64, (int64_t)na, st);
  if (rc == DWF_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = dwf_cuda_check(c, e, "coarse_build");
  }
  if (rc) {
    coarse_destroy(C);
    return rc;
  }
  *out = C;
  return DWF_OK;
}

extern "C" int coarse_destroy(dwf_coarse* C) {
  if (!C) return DWF_OK;
  if (C->A64) cudaFree(C->A64);
  if (C->A32) cudaFree(C->A32);
  if (C->At) cudaFree(C->At);
  if (C->At4) cudaFree(C->At4);
  if (C->Bt) cudaFree(C->Bt);
  if (C->Arb) cudaFree(C->Arb);
  coarse_defl_free(C);
  if (C->err) cudaFree(C->err);
  if (C->err_host) cudaFreeHost(C->err_host);
  if (C->err_ready) cudaEventDestroy(C->err_ready);
  for (int i = 0; i < 6; i++)
    if (C->ws[i]) cudaFree(C->ws[i]);
  delete C;
  return DWF_OK;
}

extern "C" int coarse_export(const dwf_coarse* C, void* A, int* dims) {
  if (!C) return DWF_EINVAL;
  if (dims) {
    for (int m = 0; m < 4; m++) dims[m] = C->g.Lc[m];
    dims[4] = C->nb;
  }
  if (A) {
    const size_t na = (size_t)C->g.nc * 9 * C->nb * C->nb;
    if (cudaMemcpy(A, C->A64, na * sizeof(double2), cudaMemcpyDefault) != cudaSuccess) {
      cudaGetLastError();
      return DWF_ECUDA;
    }
  }
  return DWF_OK;
}

extern "C" int coarse_apply(dwf_coarse* C, void* out, const void* in, int nrhs, int prec, void* stream) {
  if (!C || !out || !in || nrhs < 1) return DWF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  dwf_ctx* c = C->ctx;
  if (prec == DWF_F32) {
    int rc = coarse_apply_dev(C, (float2*)out, (const float2*)in, nrhs, st);
    if (rc) return rc;
    DWF_CUDA(c, cudaGetLastError());
    return DWF_OK;
  }
  if (prec != DWF_TF32) return dwf_fail(c, DWF_EINVAL, "coarse_apply precision: DWF_F32 or DWF_TF32");
  if (((uintptr_t)out & 15) || ((uintptr_t)in & 15)) return dwf_fail(c, DWF_EINVAL, "alignment");
  if (!C->err) {
    if (cudaMalloc(&C->err, sizeof(int)) != cudaSuccess || cudaMallocHost(&C->err_host, sizeof(int)) != cudaSuccess ||
        cudaEventCreateWithFlags(&C->err_ready, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return dwf_fail(c, DWF_ENOMEM, "coarse error flag");
    }
    *C->err_host = 0;
    DWF_CUDA(c, cudaMemsetAsync(C->err, 0, sizeof(int), st));
    DWF_CUDA(c, cudaEventRecord(C->err_ready, st));
  }
  // The kernel's bounded waits report through a sticky device flag that is
  // copied to pinned host memory after every apply; a flag raised by an
  // earlier apply whose copy has landed is returned here, without waiting.
  if (cudaEventQuery(C->err_ready) == cudaSuccess && *C->err_host) {
    *C->err_host = 0;
    DWF_CUDA(c, cudaMemsetAsync(C->err, 0, sizeof(int), st));
    return dwf_fail(c, DWF_ETIMEOUT, "tensor-core coarse apply: a bounded barrier wait gave up (earlier call)");
  }
  cudaGetLastError();  // cudaEventQuery's cudaErrorNotReady is not an error
  int rc = coarse_apply_tc(c, (float2*)out, (const float2*)in, C->A32, &C->At, &C->At4, &C->Bt, &C->Bt_bytes, C->nb,
                           C->g.nc, C->g.Lc, nrhs, C->err, st);
  if (rc == DWF_EINVAL)
    return dwf_fail(c, rc, "tensor-core coarse apply needs nb = 32, an even number of coarse sites, nrhs 16/32/64");
  if (rc) return dwf_fail(c, rc, "tensor-core coarse apply");
  DWF_CUDA(c, cudaMemcpyAsync(C->err_host, C->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DWF_CUDA(c, cudaEventRecord(C->err_ready, st));
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

extern "C" int coarse_apply_status(dwf_coarse* C, void* stream) {
  if (!C) return DWF_EINVAL;
  dwf_ctx* c = C->ctx;
  DWF_CUDA(c, cudaStreamSynchronize((cudaStream_t)stream));
  if (!C->err_host) return DWF_OK;
  DWF_CUDA(c, cudaEventSynchronize(C->err_ready));
  if (*C->err_host) {
    *C->err_host = 0;
    DWF_CUDA(c, cudaMemsetAsync(C->err, 0, sizeof(int), (cudaStream_t)stream));
    DWF_CUDA(c, cudaStreamSynchronize((cudaStream_t)stream));
    return dwf_fail(c, DWF_ETIMEOUT, "tensor-core coarse apply: a bounded barrier wait gave up");
  }
  return DWF_OK;
}

extern "C" int coarse_solve(dwf_coarse* C, void* e, const void* r, double tol, int maxiter, int* iters,
                            void* stream) {
  if (!C || !e || !r || !(tol > 0) || maxiter < 1) return DWF_EINVAL;
  int it = 0;
  int rc = coarse_cg(C, (float2*)e, (const float2*)r, tol, maxiter, &it, (cudaStream_t)stream);
  if (iters) *iters = it;
  if (rc) return rc;
  DWF_CUDA(C->ctx, cudaStreamSynchronize((cudaStream_t)stream));
  return DWF_OK;
}

extern "C" int coarse_solve_rb(dwf_coarse* C, void* e, const void* r, double tol, int maxiter, int* iters,
                               void* stream) {
  if (!C || !e || !r || !(tol > 0) || maxiter < 1) return DWF_EINVAL;
  int it = 0;
  int rc = coarse_rbcg(C, (float2*)e, (const float2*)r, tol, maxiter, &it, (cudaStream_t)stream);
  if (iters) *iters = it;
  if (rc) return rc;
  DWF_CUDA(C->ctx, cudaStreamSynchronize((cudaStream_t)stream));
  return DWF_OK;
}

extern "C" int dwf_restrict(dwf_ctx* c, void* out, const void* in, const void* basis, int nb, const int block[4],
                            int nrhs, int prec, void* stream) {
  if (!c || !out || !in || !basis || !block) return DWF_EINVAL;
  BlockGeom g;
  int rc = make_geom(c, block, &g);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  double2* tmp = (double2*)ws(c, MW_T11 + 0, (size_t)g.nc * nb * nrhs * sizeof(double2));
  if (!tmp) return dwf_fail(c, DWF_ENOMEM, "workspace");
  rc = block_inner(c, g, basis, nb, in, nrhs, prec, tmp, (long long)nb * nrhs, nrhs, 0, 0, st);
  if (rc) return rc;
  rc = blas_copy(c, out, DWF_F32, tmp, DWF_F64, (int64_t)g.nc * nb * nrhs, st);
  if (rc) return rc;
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

extern "C" int dwf_prolong(dwf_ctx* c, void* out, const void* in, const void* basis, int nb, const int block[4],
                           int nrhs, int prec, int accumulate, void* stream) {
  if (!c || !out || !in || !basis || !block) return DWF_EINVAL;
  BlockGeom g;
  int rc = make_geom(c, block, &g);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  double2* tmp = (double2*)ws(c, MW_T11 + 0, (size_t)g.nc * nb * nrhs * sizeof(double2));
  if (!tmp) return dwf_fail(c, DWF_ENOMEM, "workspace");
  rc = blas_copy(c, tmp, DWF_F64, in, DWF_F32, (int64_t)g.nc * nb * nrhs, st);
  if (rc) return rc;
  rc = block_combine(c, g, out, nrhs, prec, basis, nb, prec, tmp, (long long)nb * nrhs, nrhs, accumulate, st);
  if (rc) return rc;
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

// ---------------------------------------------------------------------- MG setup / solve
namespace {

// Chebyshev smoother S_cheb([a,b],N) of Eq. (24) with M = M^dag = H_DW:
// z = [c0/2 + sum_{j=1}^{N-1} c_j T_j(y(H^2))] H r.  FP32 full fields.
int smoother(dwf_mg* G, void* z, const void* r, cudaStream_t st, double* nH) {
  dwf_ctx* c = G->ctx;
  const int64_t n = full_elems(c);
  const size_t bytes = n * sizeof(float2);
  void* v = ws(c, MW_T0, bytes);
  void* tp = ws(c, MW_T1, bytes);
  void* tc = ws(c, MW_T2, bytes);
  void* ax = ws(c, MW_T3, bytes);
  void* tmp = ws(c, MW_T4, bytes);
  if (!v || !tp || !tc || !ax || !tmp) return dwf_fail(c, DWF_ENOMEM, "smoother workspace");
  const double a = G->p.smooth_lo, b = G->p.smooth_hi;
  const int N = G->p.smooth_order;
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
  const double mf[1] = {G->p.mf};
  int rc = ddw_apply(c, v, r, mf, 0, 1, DWF_F32, 1, st);  // v = H r
  if (rc) return rc;
  *nH += 1;
  rc = blas_axpby(c, 0.5 * cf[0], v, DWF_F32, 0.0, z, DWF_F32, n, st);
  if (rc) return rc;
  if (N < 2) return DWF_OK;
  const double xa = 2.0 / (b - a), xb = -(b + a) / (b - a);
  rc = blas_copy(c, tp, DWF_F32, v, DWF_F32, n, st);
  if (rc) return rc;
  rc = hsq(c, ax, tp, tmp, G->p.mf, DWF_F32, 1, st);
  if (rc) return rc;
  *nH += 2;
  rc = blas_axpbypcz(c, xa, ax, xb, tp, 0.0, tc, n, DWF_F32, st);  // T1
  if (rc) return rc;
  rc = blas_axpby(c, cf[1], tc, DWF_F32, 1.0, z, DWF_F32, n, st);
  if (rc) return rc;
  for (int j = 2; j < N; j++) {
    // tp <- T_j, z += c_j T_j: the recurrence step fused into the last hops of H^2
    const ChebFuse fz = {tc, tp, z, 2 * xa, 2 * xb, cf[j]};
    rc = hsq(c, ax, tc, tmp, G->p.mf, DWF_F32, 1, st, &fz);
    if (rc) return rc;
    *nH += 2;
    void* t = tp;
    tp = tc;
    tc = t;
  }
  return DWF_OK;
}

// V(1,1) of Eqs. (26)-(28) on residual r0 with x0 = 0: x1 = S r0, r1 = r0 - H x1,
// x2 = x1 + P A^-1 P^dag r1, r2 = r0 - H x2, x3 = x2 + S r2.  FP32.
// The HDCR coarse correction x += P A^-1 P^dag r1 (block restriction, coarse
// solve, block prolongation).
int coarse_correction(dwf_mg* G, void* x, const void* rr, cudaStream_t st, int* ncoarse) {
  dwf_ctx* c = G->ctx;
  dwf_coarse* C = G->coarse;
  int rc = DWF_OK;
  const int64_t ncv = (int64_t)C->g.nc * C->nb;
  double2* t64 = (double2*)ws(c, MW_T7, ncv * sizeof(double2));
  void *rc32, *ec32;
  if (!t64 || (rc = coarse_ws(C, 5, 2 * ncv * sizeof(float2), &rc32))) return rc ? rc : dwf_fail(c, DWF_ENOMEM, "ws");
  ec32 = (float2*)rc32 + ncv;
  rc = block_inner(c, C->g, G->basis, C->nb, rr, 1, DWF_F32, t64, C->nb, 1, 0, 0, st);  // P^dag r1
  if (rc) return rc;
  rc = blas_copy(c, rc32, DWF_F32, t64, DWF_F64, ncv, st);
  if (rc) return rc;
  int it = 0;
  rc = G->p.coarse_solver == DWF_COARSE_RB
           ? coarse_rbcg(C, (float2*)ec32, (const float2*)rc32, G->p.coarse_tol, G->p.coarse_maxiter, &it, st)
           : coarse_cg(C, (float2*)ec32, (const float2*)rc32, G->p.coarse_tol, G->p.coarse_maxiter, &it, st);
  if (rc) return rc;
  *ncoarse += it;
  rc = blas_copy(c, t64, DWF_F64, ec32, DWF_F32, ncv, st);
  if (rc) return rc;
  return block_combine(c, C->g, x, 1, DWF_F32, G->basis, C->nb, DWF_F32, t64, C->nb, 1, 1, st);
}

int vcycle(dwf_mg* G, void* x, const void* r0, cudaStream_t st, double* nH, int* ncoarse) {
  dwf_ctx* c = G->ctx;
  const int64_t n = full_elems(c);
  const size_t bytes = n * sizeof(float2);
  void* rr = ws(c, MW_T5, bytes);
  void* s2 = ws(c, MW_T6, bytes);
  if (!rr || !s2) return dwf_fail(c, DWF_ENOMEM, "vcycle workspace");
  const double mf[1] = {G->p.mf};
  int rc = smoother(G, x, r0, st, nH);
  if (rc) return rc;
  rc = ddw_apply(c, rr, x, mf, 0, 1, DWF_F32, 1, st);
  if (rc) return rc;
  *nH += 1;
  rc = blas_axpby(c, 1.0, r0, DWF_F32, -1.0, rr, DWF_F32, n, st);  // r1
  if (rc) return rc;
  // x2 = x1 + P e: the HDCR coarse solve, or the hybrid levels (Algorithm F)
  rc = G->hyb ? hybrid_correction(G->hyb, x, rr, st, ncoarse) : coarse_correction(G, x, rr, st, ncoarse);
  if (rc) return rc;
  rc = ddw_apply(c, rr, x, mf, 0, 1, DWF_F32, 1, st);
  if (rc) return rc;
  *nH += 1;
  rc = blas_axpby(c, 1.0, r0, DWF_F32, -1.0, rr, DWF_F32, n, st);  // r2
  if (rc) return rc;
  rc = smoother(G, s2, rr, st, nH);
  if (rc) return rc;
  return blas_axpby(c, 1.0, s2, DWF_F32, 1.0, x, DWF_F32, n, st);  // x3
}

// One V(1,1) application replayed from a CUDA graph.  Its launch sequence
// (the two smoothers' hopping and Chebyshev launches, the restriction, one
// cooperative coarse-CG launch, the prolongation) is captured once per solve
// on a private stream, after a plain warm-up V-cycle has sized every
// workspace, and replayed for each pGCR direction; the residual is copied
// into, and the direction out of, two fixed buffers.  The coarse CG then runs
// without host synchronisation and reports its iteration count and any error
// through a device accumulator that the solve reads at its next
// synchronisation.  The graph lives for one mg_solve call, so no workspace
// can move under it.
struct VGraph {
  dwf_ctx* c = nullptr;
  cudaStream_t gs = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* in = nullptr;
  void* out = nullptr;
  int* acc = nullptr;    // device [coarse iterations, error bits]
  int* acc_h = nullptr;  // pinned mirror
  int64_t launches = 0;  // kernel launches per replay
  double nH = 0;         // H_DW applications per replay
  int state = 0;         // 0: not built, 1: ready, -1: not available
  int replays = 0;
  ~VGraph() {
    if (gs) cudaStreamSynchronize(gs);
    if (exec) cudaGraphExecDestroy(exec);
    if (gs) cudaStreamDestroy(gs);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (in) cudaFree(in);
    if (out) cudaFree(out);
    if (acc) cudaFree(acc);
    if (acc_h) cudaFreeHost(acc_h);
  }
};

int vgraph_build(VGraph& V, dwf_mg* G, cudaStream_t st) {
  dwf_ctx* c = G->ctx;
  V.c = c;
  V.state = -1;
  const size_t bytes = (size_t)full_elems(c) * sizeof(float2);
  if (cudaStreamCreateWithFlags(&V.gs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&V.e0, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&V.e1, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(&V.in, bytes) != cudaSuccess || cudaMalloc(&V.out, bytes) != cudaSuccess ||
      cudaMalloc(&V.acc, 2 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&V.acc_h, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return DWF_OK;  // plain launches
  }
  V.acc_h[0] = V.acc_h[1] = 0;
  DWF_CUDA(c, cudaMemsetAsync(V.acc, 0, 2 * sizeof(int), st));
  DWF_CUDA(c, cudaStreamSynchronize(st));
  const int64_t l0 = c->launches;
  double nH = 0;
  int nco = 0;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(V.gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return DWF_OK;
  }
  G->coarse->cg_acc = V.acc;
  const std::string err_before = c->err;
  const int rc = vcycle(G, V.out, V.in, V.gs, &nH, &nco);
  G->coarse->cg_acc = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(V.gs, &graph);
  V.launches = c->launches - l0;
  c->launches = l0;
  if (rc || ec != cudaSuccess || !graph || cudaGraphInstantiate(&V.exec, graph, 0) != cudaSuccess) {
    // capture not possible (e.g. a launch form the CUDA driver cannot record):
    // the solve continues with plain launches
    if (graph) cudaGraphDestroy(graph);
    V.exec = nullptr;
    c->err = err_before;
    cudaGetLastError();
    return DWF_OK;
  }
  cudaGraphDestroy(graph);
  V.nH = nH;
  V.state = 1;
  return DWF_OK;
}

int vgraph_run(VGraph& V, void* z, const void* r, cudaStream_t st, double* nH) {
  dwf_ctx* c = V.c;
  const size_t bytes = (size_t)full_elems(c) * sizeof(float2);
  DWF_CUDA(c, cudaMemcpyAsync(V.in, r, bytes, cudaMemcpyDeviceToDevice, st));
  DWF_CUDA(c, cudaEventRecord(V.e0, st));
  DWF_CUDA(c, cudaStreamWaitEvent(V.gs, V.e0, 0));
  DWF_CUDA(c, cudaGraphLaunch(V.exec, V.gs));
  DWF_CUDA(c, cudaEventRecord(V.e1, V.gs));
  DWF_CUDA(c, cudaStreamWaitEvent(st, V.e1, 0));
  DWF_CUDA(c, cudaMemcpyAsync(z, V.out, bytes, cudaMemcpyDeviceToDevice, st));
  DWF_CUDA(c, cudaMemcpyAsync(V.acc_h, V.acc, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  c->launches += V.launches;
  *nH += V.nH;
  V.replays++;
  return DWF_OK;
}

// Error bits of the graph's coarse CG, valid after a synchronisation.
int vgraph_check(const VGraph& V) {
  if (V.state != 1 || !V.acc_h[1]) return DWF_OK;
  return dwf_fail(V.c, (V.acc_h[1] & 1) ? DWF_ETIMEOUT : DWF_ENAN,
                  (V.acc_h[1] & 1) ? "coarse CG grid barrier timed out" : "NaN in coarse solve");
}

}  // namespace

extern "C" int mg_setup(dwf_ctx* c, const dwf_mg_params* p, const void* eta, dwf_mg** out, void* stream) {
  Timer timer;
  if (!c || !p || !eta || !out) return DWF_EINVAL;
  *out = nullptr;
  const int nb = p->nbasis;
  if (nb < 2 || (nb & 1) || nb > 64 || nb / 2 > 32) return dwf_fail(c, DWF_EINVAL, "nbasis must be even, <= 64");
  if (p->subspace_mode != DWF_SUBSPACE_BATCH && p->subspace_mode != DWF_SUBSPACE_RECURSIVE)
    return dwf_fail(c, DWF_EINVAL, "bad subspace mode");
  if (p->coarse_solver != DWF_COARSE_CG && p->coarse_solver != DWF_COARSE_RB &&
      p->coarse_solver != DWF_COARSE_DEFLATED)
    return dwf_fail(c, DWF_EINVAL, "bad coarse solver");
  dwf_mg* G = new (std::nothrow) dwf_mg();
  if (!G) return DWF_ENOMEM;
  G->ctx = c;
  G->p = *p;
  int rc = make_geom(c, p->block, &G->g);
  if (rc) {
    delete G;
    return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = full_elems(c);
  const int nplus = nb / 2;
  // Memory: the basis (nb FP32 full fields) is the only field-sized storage
  // the setup keeps; the filter writes into it, the chirality projection and
  // the orthonormalisation work on it in place, and the coarse build takes its
  // H_DW images eight vectors at a time.
  if (cudaMalloc(&G->basis, (size_t)n * nb * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    mg_destroy(G);
    return dwf_fail(c, DWF_ENOMEM, "mg basis");
  }
  float2* B = G->basis;
  // 1. filtered vectors: batch mode filters nb Gaussians (eight at a time);
  //    recursive mode builds nb/2 vectors from one Gaussian.
  double lmax = p->lambda_max;
  const int chunk = 8;
  if (p->subspace_mode == DWF_SUBSPACE_BATCH) {
    void* e32 = ws(c, MW_T10, (size_t)n * chunk * sizeof(float2));
    rc = e32 ? DWF_OK : dwf_fail(c, DWF_ENOMEM, "ws");
    for (int r0 = 0; r0 < nb && rc == DWF_OK; r0 += chunk) {
      const int nr = nb - r0 < chunk ? nb - r0 : chunk;
      rc = blas_copy(c, e32, DWF_F32, (const double2*)eta + (size_t)r0 * n, DWF_F64, n * nr, st);
      if (rc == DWF_OK)
        rc = filter_core(c, B + (size_t)r0 * n, e32, nr, p->lambda_lo, lmax, p->filter_order, p->mf, DWF_F32, true,
                         st);
    }
    if (rc == DWF_OK) rc = normalise_fields(c, B, nb, n, DWF_F32, st);
  } else {
    void* e32 = ws(c, MW_T10, (size_t)n * sizeof(float2));
    rc = e32 ? blas_copy(c, e32, DWF_F32, eta, DWF_F64, n, st) : dwf_fail(c, DWF_ENOMEM, "ws");
    if (rc == DWF_OK)
      rc = cheby_recursive_basis(c, B, e32, p->lambda_lo, lmax, p->filter_order, p->delta, nplus, p->mf, DWF_F32,
                                 stream);
  }
  // 2. chirality projection in place: the first nb/2 basis vectors take +, the rest -
  if (rc == DWF_OK) {
    if (p->subspace_mode == DWF_SUBSPACE_BATCH) {
      rc = chiral(c, B, B, +1, DWF_F32, nplus, st);
      if (rc == DWF_OK) rc = chiral(c, B + (size_t)nplus * n, B + (size_t)nplus * n, -1, DWF_F32, nplus, st);
    } else {
      rc = chiral(c, B + (size_t)nplus * n, B, -1, DWF_F32, nplus, st);
      if (rc == DWF_OK) rc = chiral(c, B, B, +1, DWF_F32, nplus, st);
    }
  }
  // 3. block orthonormalisation in place: Cholesky-QR twice per block and
  //    chirality, Gram matrices, factorisation and updates in FP64 arithmetic
  if (rc == DWF_OK) rc = ortho_inplace_f32(c, G->g, B, nb, nplus, st);
  if (rc == DWF_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = dwf_cuda_check(c, e, "mg_setup");
  }
  G->setup_seconds = timer.sec();
  // 4. little Dirac operator of H_DW from the FP32 basis
  Timer t2;
  if (rc == DWF_OK) rc = coarse_build(c, G->basis, nb, nplus, p->block, p->mf, DWF_F32, &G->coarse, stream);
  if (rc == DWF_OK && p->coarse_solver == DWF_COARSE_RB) rc = coarse_rb_ready(G->coarse, st);
  if (rc == DWF_OK && p->coarse_solver == DWF_COARSE_DEFLATED) {
    // Lanczos start vector: the restriction of the first eta (the setup's
    // own random input)
    const int64_t ncv = (int64_t)G->g.nc * nb;
    double2* t64 = (double2*)ws(c, MW_T7, ncv * sizeof(double2));
    void* e1 = ws(c, MW_T10, (size_t)n * sizeof(float2));
    void* v0 = nullptr;
    rc = (!t64 || !e1) ? dwf_fail(c, DWF_ENOMEM, "ws") : coarse_ws(G->coarse, 4, ncv * sizeof(float2), &v0);
    if (rc == DWF_OK) rc = blas_copy(c, e1, DWF_F32, eta, DWF_F64, n, st);
    if (rc == DWF_OK) rc = block_inner(c, G->g, B, nb, e1, 1, DWF_F32, t64, nb, 1, 0, 0, st);
    if (rc == DWF_OK) rc = blas_copy(c, v0, DWF_F32, t64, DWF_F64, ncv, st);
    if (rc == DWF_OK)
      rc = coarse_deflate(G->coarse, v0, p->coarse_nev, p->coarse_lanczos, p->coarse_cheb_order, p->coarse_cheb_lo,
                          0.0, nullptr, stream);
  }
  G->coarse_op_seconds = t2.sec();
  G->lambda_max_used = lmax;
  // the field-sized setup workspaces are released for the solve
  if (rc == DWF_OK) {
    DWF_CUDA(c, cudaStreamSynchronize(st));
    for (int slot = MW_T0; slot <= MW_T11; slot++) dwf_ws_release(c, slot);
  }
  if (rc) {
    mg_destroy(G);
    return rc;
  }
  *out = G;
  return DWF_OK;
}

extern "C" int mg_destroy(dwf_mg* G) {
  if (!G) return DWF_OK;
  if (G->basis) cudaFree(G->basis);
  if (G->coarse) coarse_destroy(G->coarse);
  if (G->hyb) hybrid_free(G->hyb);
  delete G;
  return DWF_OK;
}

// Algorithm F: the fine level of mg_solve (pGCR, V(1,1) with the Chebyshev
// smoother on H_DW) over the hybrid levels built by hybrid.cu.
extern "C" int mg_setup_hybrid(dwf_ctx* c, const dwf_mg_params* p, const dwf_hybrid_params* hp, const void* eta4,
                               const void* eta1, dwf_mg** out, void* stream) {
  if (!c || !p || !hp || !eta4 || !eta1 || !out) return DWF_EINVAL;
  *out = nullptr;
  if (p->coarse_solver != DWF_COARSE_CG && p->coarse_solver != DWF_COARSE_RB &&
      p->coarse_solver != DWF_COARSE_DEFLATED)
    return dwf_fail(c, DWF_EINVAL, "bad coarse solver");
  if (p->smooth_order < 1 || !(p->smooth_hi > p->smooth_lo && p->smooth_lo > 0))
    return dwf_fail(c, DWF_EINVAL, "bad smoother");
  dwf_mg* G = new (std::nothrow) dwf_mg();
  if (!G) return DWF_ENOMEM;
  G->ctx = c;
  G->p = *p;
  G->p.no_graph = 1;  // the level-1 GCR reads its scalars on the host
  G->p.nbasis = 0;
  int rc = hybrid_build(c, p, hp, eta4, eta1, &G->hyb, (cudaStream_t)stream);
  if (rc) {
    delete G;
    return rc;
  }
  G->setup_seconds = hybrid_setup_seconds(G->hyb);
  G->coarse_op_seconds = hybrid_coarse_seconds(G->hyb);
  G->lambda_max_used = hp->lambda_max4;
  *out = G;
  return DWF_OK;
}

extern "C" int mg_hybrid_export(const dwf_mg* G, int what, void* out) {
  if (!G || !out) return DWF_EINVAL;
  if (!G->hyb) return dwf_fail(G->ctx, DWF_EINVAL, "not a hybrid setup");
  return hybrid_export(G->hyb, what, out);
}

extern "C" int mg_hybrid_level1(dwf_mg* G, int op, void* out, const void* in, int nvec, void* stream) {
  if (!G || !out || !in) return DWF_EINVAL;
  if (!G->hyb) return dwf_fail(G->ctx, DWF_EINVAL, "not a hybrid setup");
  if (out == in) return dwf_fail(G->ctx, DWF_EINVAL, "out must not alias in");
  int rc = hybrid_level1_op(G->hyb, op, out, in, nvec, (cudaStream_t)stream);
  if (rc) return rc;
  DWF_CUDA(G->ctx, cudaGetLastError());
  return DWF_OK;
}

extern "C" int mg_export_basis(const dwf_mg* G, void* out) {
  if (!G || !out) return DWF_EINVAL;
  if (G->hyb) return dwf_fail(G->ctx, DWF_EINVAL, "hybrid setup: mg_hybrid_export");
  const size_t bytes = (size_t)full_elems(G->ctx) * G->p.nbasis * sizeof(float2);
  if (cudaMemcpy(out, G->basis, bytes, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    return DWF_ECUDA;
  }
  return DWF_OK;
}

extern "C" dwf_coarse* mg_coarse(dwf_mg* G) { return G ? (G->hyb ? hybrid_coarse(G->hyb) : G->coarse) : nullptr; }

extern "C" int mg_precondition(dwf_mg* G, void* out, const void* in, void* stream) {
  if (!G || !out || !in) return DWF_EINVAL;
  double nH = 0;
  int nc = 0;
  int rc = vcycle(G, out, in, (cudaStream_t)stream, &nH, &nc);
  if (rc) return rc;
  DWF_CUDA(G->ctx, cudaStreamSynchronize((cudaStream_t)stream));
  return DWF_OK;
}

extern "C" int mg_smooth(dwf_mg* G, void* out, const void* in, void* stream) {
  if (!G || !out || !in) return DWF_EINVAL;
  double nH = 0;
  int rc = smoother(G, out, in, (cudaStream_t)stream, &nH);
  if (rc) return rc;
  DWF_CUDA(G->ctx, cudaStreamSynchronize((cudaStream_t)stream));
  return DWF_OK;
}

// Flexible GCR(nkrylov) on H_DW x = Gamma_5 b with the V(1,1) preconditioner;
// x and the true residual in FP64, directions in FP32.
extern "C" int mg_solve(dwf_mg* G, void* x, const void* b, double tol, dwf_solve_stats* stats, void* stream) {
  Timer timer;
  if (!G || !x || !b || !(tol > 0)) return DWF_EINVAL;
  dwf_ctx* c = G->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = full_elems(c);
  const int nk = G->p.nkrylov > 0 ? G->p.nkrylov : 8;
  dwf_solve_stats S;
  memset(&S, 0, sizeof(S));
  const bool host_b = !dwf_is_device_ptr(b), host_x = !dwf_is_device_ptr(x);
  void* db = (void*)b;
  void* dx = x;
  if (host_b) {
    db = ws(c, WS_B, n * 16);
    if (!db) return dwf_fail(c, DWF_ENOMEM, "ws");
    DWF_CUDA(c, cudaMemcpyAsync(db, b, n * 16, cudaMemcpyHostToDevice, st));
  }
  if (host_x) {
    dx = ws(c, WS_X, n * 16);
    if (!dx) return dwf_fail(c, DWF_ENOMEM, "ws");
  }
  void* rhs = ws(c, WS_FULL, n * 16);                // Gamma_5 b (FP64)
  void* r64 = ws(c, WS_BP, n * 16);                  // FP64 residual
  void* t64 = ws(c, WS_RHS, n * 16);                 // FP64 temporary
  void* r32 = ws(c, WS_XLO, n * 8);                  // FP32 residual
  void* zs = ws(c, WS_RLO, (size_t)n * 8 * nk);      // directions
  void* wsv = ws(c, WS_P, (size_t)n * 8 * nk);       // H directions
  if (!rhs || !r64 || !t64 || !r32 || !zs || !wsv) return dwf_fail(c, DWF_ENOMEM, "mg_solve workspace");
  const double mf[1] = {G->p.mf};
  int rc = chiral(c, rhs, db, 1, DWF_F64, 1, st);  // placeholder overwritten below
  if (rc) return rc;
  // rhs = Gamma_5 b = (P_+ - P_-) b: 2 * (1+G5)/2 b - b
  rc = blas_axpby(c, 2.0, rhs, DWF_F64, 0.0, rhs, DWF_F64, n, st);
  if (rc) return rc;
  rc = blas_axpby(c, -1.0, db, DWF_F64, 1.0, rhs, DWF_F64, n, st);
  if (rc) return rc;
  rc = norm2_dev(c, rhs, n, DWF_F64, S_TMP0, st);
  if (rc) return rc;
  rc = read_scalars(c, S_TMP0, 1, st);
  if (rc) return rc;
  const double bnorm = sqrt(c->hscal[S_TMP0]);
  DWF_CUDA(c, cudaMemsetAsync(dx, 0, n * 16, st));
  double nH = 0;
  int ncoarse = 0;
  if (!(bnorm > 0)) {
    if (host_x) DWF_CUDA(c, cudaMemcpyAsync(x, dx, n * 16, cudaMemcpyDeviceToHost, st));
    DWF_CUDA(c, cudaStreamSynchronize(st));
    if (stats) *stats = S;
    return bnorm == 0 ? DWF_OK : dwf_fail(c, DWF_ENAN, "source is not finite");
  }
  rc = blas_copy(c, r64, DWF_F64, rhs, DWF_F64, n, st);
  if (rc) return rc;
  double res = 1.0;
  int it = 0;
  const int maxit = G->p.maxiter > 0 ? G->p.maxiter : 1000;
  bool done = false;
  std::vector<double> wnorm(nk);
  VGraph V;
  while (!done && it < maxit) {
    rc = blas_copy(c, r32, DWF_F32, r64, DWF_F64, n, st);
    if (rc) return rc;
    int k = 0;
    for (; k < nk && it < maxit; k++) {
      float2* z = (float2*)zs + (size_t)k * n;
      float2* w = (float2*)wsv + (size_t)k * n;
      if (V.state == 1) {
        rc = vgraph_run(V, z, r32, st, &nH);
      } else {
        rc = vcycle(G, z, r32, st, &nH, &ncoarse);
        if (!rc && V.state == 0 && !G->p.no_graph) rc = vgraph_build(V, G, st);
      }
      if (rc) return rc;
      rc = ddw_apply(c, w, z, mf, 0, 1, DWF_F32, 1, st);
      if (rc) return rc;
      nH += 1;
      for (int j = 0; j < k; j++) {  // orthogonalise against earlier H-directions
        const float2* wj = (const float2*)wsv + (size_t)j * n;
        const float2* zj = (const float2*)zs + (size_t)j * n;
        int np = 0;
        rc = blas_cdot_partials(c, wj, w, n, DWF_F32, st, &np);
        if (rc) return rc;
        rc = blas_finalize(c, np, 2, S_TMP0, st);
        if (rc) return rc;
        rc = read_scalars(c, S_TMP0, 2, st);
        if (rc) return rc;
        const double br = c->hscal[S_TMP0] / wnorm[j], bi = c->hscal[S_TMP0 + 1] / wnorm[j];
        rc = blas_caxpy(c, -br, -bi, wj, DWF_F32, w, DWF_F32, n, st);
        if (rc) return rc;
        rc = blas_caxpy(c, -br, -bi, zj, DWF_F32, z, DWF_F32, n, st);
        if (rc) return rc;
      }
      int np = 0;
      rc = blas_cdot_partials(c, w, r32, n, DWF_F32, st, &np);
      if (rc) return rc;
      rc = blas_finalize(c, np, 2, S_TMP0, st);
      if (rc) return rc;
      rc = norm2_dev(c, w, n, DWF_F32, S_TMP2, st);
      if (rc) return rc;
      rc = read_scalars(c, S_TMP0, 3, st);
      if (rc) return rc;
      const double ww = c->hscal[S_TMP2];
      if (!(ww > 0) || !isfinite(ww)) return dwf_fail(c, DWF_ENAN, "GCR breakdown");
      wnorm[k] = ww;
      const double ar = c->hscal[S_TMP0] / ww, ai = c->hscal[S_TMP0 + 1] / ww;
      rc = blas_caxpy(c, ar, ai, z, DWF_F32, dx, DWF_F64, n, st);
      if (rc) return rc;
      rc = blas_caxpy(c, -ar, -ai, w, DWF_F32, r32, DWF_F32, n, st);
      if (rc) return rc;
      rc = norm2_dev(c, r32, n, DWF_F32, S_TMP2, st);
      if (rc) return rc;
      rc = read_scalars(c, S_TMP2, 1, st);
      if (rc) return rc;
      rc = vgraph_check(V);
      if (rc) return rc;
      it++;
      if (sqrt(c->hscal[S_TMP2]) / bnorm <= tol) {
        k++;
        break;
      }
    }
    // restart: true residual in FP64
    rc = ddw_apply(c, t64, dx, mf, 0, 1, DWF_F64, 1, st);
    if (rc) return rc;
    nH += 1;
    rc = blas_copy(c, r64, DWF_F64, rhs, DWF_F64, n, st);
    if (rc) return rc;
    rc = blas_axpby(c, -1.0, t64, DWF_F64, 1.0, r64, DWF_F64, n, st);
    if (rc) return rc;
    rc = norm2_dev(c, r64, n, DWF_F64, S_TMP2, st);
    if (rc) return rc;
    rc = read_scalars(c, S_TMP2, 1, st);
    if (rc) return rc;
    res = sqrt(c->hscal[S_TMP2]) / bnorm;
    if (!isfinite(res)) return dwf_fail(c, DWF_ENAN, "NaN in MG solve");
    done = res <= tol;
  }
  if (host_x) DWF_CUDA(c, cudaMemcpyAsync(x, dx, n * 16, cudaMemcpyDeviceToHost, st));
  DWF_CUDA(c, cudaStreamSynchronize(st));
  rc = vgraph_check(V);
  if (rc) return rc;
  S.iterations = it;
  S.coarse_iterations = ncoarse + (V.state == 1 ? V.acc_h[0] : 0);
  S.graph_replays = V.replays;
  S.fine_matmuls = nH;
  S.true_residual = res;
  S.seconds = timer.sec();
  S.setup_seconds = G->setup_seconds;
  S.coarse_op_seconds = G->coarse_op_seconds;
  S.status = done ? DWF_OK : DWF_ENOCONV;
  if (stats) *stats = S;
  if (!done) return dwf_fail(c, DWF_ENOCONV, "mg_solve: maxiter reached before tol");
  return DWF_OK;
}
