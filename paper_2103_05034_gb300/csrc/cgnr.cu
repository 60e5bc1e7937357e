// Unpreconditioned CGNR on the full lattice (the baseline row of the paper's
// Krylov comparison, Sec. 5.1: CG on D_DW^dag D_DW x = D_DW^dag b without the
// red-black Schur complement), FP64 throughout.  Every operator application
// is two half-lattice hopping launches with the fused M5 / mf epilogue
// (D_DW, then D_DW^dag); the step lengths live in device scalars, so the host
// reads a scalar only every eight iterations.
#include <chrono>
#include <cmath>
#include <cstring>

#include "dwf_internal.cuh"

extern "C" int cgnr_solve(dwf_ctx* c, void* x, const void* b, double mf, double tol, int maxiter,
                          dwf_solve_stats* stats, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!c) return DWF_EINVAL;
  if (!x || !b) return dwf_fail(c, DWF_EINVAL, "null argument");
  if (!(tol > 0) || maxiter < 1) return dwf_fail(c, DWF_EINVAL, "bad tol or maxiter");
  if (!std::isfinite(mf)) return dwf_fail(c, DWF_EINVAL, "mass is not finite");
  if (!dwf_is_device_ptr(x) || !dwf_is_device_ptr(b)) return dwf_fail(c, DWF_EINVAL, "device buffers required");
  if (((uintptr_t)x & 15) || ((uintptr_t)b & 15)) return dwf_fail(c, DWF_EINVAL, "alignment");
  if (x == b) return dwf_fail(c, DWF_EINVAL, "x must not alias b");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = 2 * c->g.Vh * 12 * c->g.Ls;  // complex numbers of a full field
  const size_t bytes = n * 16;
  void* r = dwf_workspace(c, WS_BE, bytes);
  void* p = dwf_workspace(c, WS_BO, bytes);
  void* t = dwf_workspace(c, WS_XE, bytes);
  void* Ap = dwf_workspace(c, WS_XO, bytes);
  if (!r || !p || !t || !Ap) return dwf_fail(c, DWF_ENOMEM, "solver workspace");
  const double m1[1] = {mf};
  dwf_solve_stats S;
  memset(&S, 0, sizeof(S));
  double matmuls = 0;  // full-lattice D_DW / D_DW^dag applications
  int rc;

  // |b|
  rc = norm2_dev(c, b, n, DWF_F64, S_TMP0, st);
  if (rc) return rc;
  rc = read_scalars(c, S_TMP0, 1, st);
  if (rc) return rc;
  const double bnorm = sqrt(c->hscal[S_TMP0]);
  DWF_CUDA(c, cudaMemsetAsync(x, 0, bytes, st));
  if (!std::isfinite(bnorm)) return dwf_fail(c, DWF_ENAN, "source is not finite");
  if (bnorm == 0) {
    DWF_CUDA(c, cudaStreamSynchronize(st));
    S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = S;
    return DWF_OK;
  }
  // true residual |b - D x| / |b| into *res (x as it stands)
  auto true_residual = [&](double* res) -> int {
    int q = ddw_apply(c, t, x, m1, 0, 0, DWF_F64, 1, st);
    if (q) return q;
    q = blas_axpby(c, 1.0, b, DWF_F64, -1.0, t, DWF_F64, n, st);
    if (q) return q;
    q = norm2_dev(c, t, n, DWF_F64, S_TMP1, st);
    if (q) return q;
    q = read_scalars(c, S_TMP1, 1, st);
    if (q) return q;
    matmuls += 1;
    *res = sqrt(c->hscal[S_TMP1]) / bnorm;
    return std::isfinite(*res) ? DWF_OK : dwf_fail(c, DWF_ENAN, "NaN in CG residual");
  };

  // r = p = D^dag b, rr = |r|^2
  rc = ddw_apply(c, r, b, m1, 1, 0, DWF_F64, 1, st);
  if (rc) return rc;
  matmuls += 1;
  rc = norm2_dev(c, r, n, DWF_F64, S_RR, st);
  if (rc) return rc;
  DWF_CUDA(c, cudaMemcpyAsync(p, r, bytes, cudaMemcpyDeviceToDevice, st));
  rc = read_scalars(c, S_RR, 1, st);
  if (rc) return rc;
  const double rhs_norm = sqrt(c->hscal[S_RR]);
  // the normal-equation residual is checked against tol_n; when it is met
  // the true residual decides, and tol_n tightens tenfold if it is not
  double tol_n = tol, res = 1.0;
  bool converged = false;
  int it = 0;
  const int check_every = 8;
  while (!converged && it < maxiter) {
    // t = D p, |t|^2 = <p, D^dag D p> -> alpha = rr / pAp
    rc = ddw_apply(c, t, p, m1, 0, 0, DWF_F64, 1, st);
    if (rc) return rc;
    int np = 0;
    rc = blas_norm2_partials(c, t, n, DWF_F64, st, &np);
    if (rc) return rc;
    rc = blas_finalize_mode(c, np, 1, S_PAP, 1, st);
    if (rc) return rc;
    // Ap = D^dag t; x += alpha p, r -= alpha Ap, |r|^2 -> beta
    rc = ddw_apply(c, Ap, t, m1, 1, 0, DWF_F64, 1, st);
    if (rc) return rc;
    rc = blas_cg_xr(c, x, r, p, Ap, n, DWF_F64, S_ALPHA, st, &np);
    if (rc) return rc;
    rc = blas_finalize_mode(c, np, 1, S_RRNEW, 2, st);
    if (rc) return rc;
    rc = blas_cg_p(c, p, r, n, DWF_F64, S_BETA, st);
    if (rc) return rc;
    matmuls += 2;
    it++;
    if (it % check_every == 0 || it == maxiter) {
      rc = read_scalars(c, S_RR, 1, st);
      if (rc) return rc;
      const double rr = c->hscal[S_RR];
      if (!std::isfinite(rr)) return dwf_fail(c, DWF_ENAN, "NaN in CG residual");
      if (sqrt(rr) <= tol_n * rhs_norm || it == maxiter) {
        rc = true_residual(&res);
        if (rc) return rc;
        converged = res <= tol;
        if (!converged) tol_n *= 0.1;
      }
    }
  }
  DWF_CUDA(c, cudaStreamSynchronize(st));
  S.iterations = it;
  S.true_residual = res;
  S.fine_matmuls = matmuls;
  S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  S.status = converged ? DWF_OK : DWF_ENOCONV;
  DWF_CUDA(c, cudaGetLastError());
  if (stats) *stats = S;
  if (!converged) return dwf_fail(c, DWF_ENOCONV, "maxiter reached before tol");
  return DWF_OK;
}
