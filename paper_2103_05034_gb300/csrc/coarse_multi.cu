// Coarse solves for many right-hand sides (the multi-RHS use of the little
// Dirac operator of Sec. 3.1, Eq. 18): CG on A^2 e_r = A rhs_r for nrhs
// independent right-hand sides at once, each with its own step lengths, so
// that every application of A covers all of them -- on the tensor cores
// (coarse_apply with DWF_TF32) or on the CUDA cores (DWF_F32).  Vectors are
// [nc][nb][nrhs] FP32 complex; scalars and sums in FP64, per right-hand side.
// The host reads the residuals every eight iterations; a right-hand side
// whose normal residual has reached tol stops changing (its step length is
// set to zero), and the call returns when all have.
#include <math.h>
#include <string.h>

#include <vector>

#include "coarse_internal.cuh"

namespace {

constexpr int MT = 256;
constexpr int MBLK = 304;  // two CTAs per SM

// part[b][r] = the sum over CTA b's rows of |v[row][r]|^2, for every
// right-hand side r (thread t takes r = t mod nrhs and every (256/nrhs)-th row).
__global__ void __launch_bounds__(MT) k_mnorm(const float2* __restrict__ v, long long rows, int nrhs, double* part) {
  __shared__ double sh[MT];
  const int r = threadIdx.x % nrhs, lane_rows = MT / nrhs, rl = threadIdx.x / nrhs;
  double acc = 0.0;
  if (rl < lane_rows)
    for (long long row = (long long)blockIdx.x * lane_rows + rl; row < rows; row += (long long)gridDim.x * lane_rows) {
      const float2 z = v[row * nrhs + r];
      acc += (double)z.x * z.x + (double)z.y * z.y;
    }
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < nrhs) {
    double s = 0.0;
    for (int k = 0; k < lane_rows; k++) s += sh[k * nrhs + threadIdx.x];
    part[(size_t)blockIdx.x * nrhs + threadIdx.x] = s;
  }
}

// Per right-hand side r (one thread each): sum the nblk partials in block
// order into dst[r], then mode 1: alpha_r = rr_r / pAp_r (0 once converged);
// mode 2: beta_r = rrnew_r / rr_r, rr_r = rrnew_r; mode 0: the sum only.
// sc layout: [0] rr, [1] pAp / rrnew, [2] alpha, [3] beta, [4] done flag, per r.
__global__ void k_mscalars(const double* part, int nblk, int nrhs, double* sc, int dst, int mode) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  double s = 0.0;
  for (int b = 0; b < nblk; b++) s += part[(size_t)b * nrhs + r];
  double* q = sc + 5 * r;
  q[dst] = s;
  if (mode == 1) {
    q[2] = (q[4] != 0.0 || !(s > 0)) ? 0.0 : q[0] / s;
  } else if (mode == 2) {
    q[3] = q[4] != 0.0 ? 0.0 : s / q[0];
    if (q[4] == 0.0) q[0] = s;
  }
}

// e_r += alpha_r p_r; r_r -= alpha_r q_r
__global__ void __launch_bounds__(MT) k_mupdate(float2* e, float2* res, const float2* __restrict__ p,
                                                const float2* __restrict__ q, long long n, int nrhs, const double* sc) {
  for (long long i = (long long)blockIdx.x * MT + threadIdx.x; i < n; i += (long long)gridDim.x * MT) {
    const float a = (float)sc[5 * (i % nrhs) + 2];
    const float2 pv = p[i], qv = q[i];
    float2 ev = e[i], rv = res[i];
    ev.x = fmaf(a, pv.x, ev.x);
    ev.y = fmaf(a, pv.y, ev.y);
    rv.x = fmaf(-a, qv.x, rv.x);
    rv.y = fmaf(-a, qv.y, rv.y);
    e[i] = ev;
    res[i] = rv;
  }
}

// p_r = r_r + beta_r p_r
__global__ void __launch_bounds__(MT) k_mdir(float2* p, const float2* __restrict__ res, long long n, int nrhs,
                                             const double* sc) {
  for (long long i = (long long)blockIdx.x * MT + threadIdx.x; i < n; i += (long long)gridDim.x * MT) {
    const float b = (float)sc[5 * (i % nrhs) + 3];
    const float2 rv = res[i], pv = p[i];
    p[i] = make_float2(fmaf(b, pv.x, rv.x), fmaf(b, pv.y, rv.y));
  }
}

unsigned mgrid(long long n) {
  long long g = (n + MT - 1) / MT;
  return (unsigned)(g > MBLK ? MBLK : (g < 1 ? 1 : g));
}

}  // namespace

extern "C" int coarse_apply(dwf_coarse* C, void* out, const void* in, int nrhs, int prec, void* stream);

extern "C" int coarse_solve_multi(dwf_coarse* C, void* e, const void* rhs, int nrhs, double tol, int maxiter,
                                  int* iters, int prec, void* stream) {
  if (!C || !e || !rhs || nrhs < 1 || nrhs > 64 || !(tol > 0) || maxiter < 1) return DWF_EINVAL;
  dwf_ctx* c = C->ctx;
  if (prec != DWF_F32 && prec != DWF_TF32) return dwf_fail(c, DWF_EINVAL, "coarse_solve_multi: DWF_F32 or DWF_TF32");
  if (MT % nrhs) return dwf_fail(c, DWF_EINVAL, "coarse_solve_multi: nrhs must divide 256");
  cudaStream_t st = (cudaStream_t)stream;
  const long long rows = (long long)C->g.nc * C->nb, n = rows * nrhs;
  void *work, *part, *scal;
  int rc;
  if ((rc = coarse_ws(C, 0, 4 * n * sizeof(float2), &work)) || (rc = coarse_ws(C, 1, (size_t)MBLK * nrhs * sizeof(double), &part)) ||
      (rc = coarse_ws(C, 2, 5 * 64 * sizeof(double), &scal)))
    return rc;
  float2 *r = (float2*)work, *p = r + n, *t = r + 2 * n, *q = r + 3 * n;
  double* sc = (double*)scal;
  double* pt = (double*)part;
  const unsigned g = mgrid(n), gr = mgrid(rows);
  auto apply = [&](float2* o, const float2* v) -> int { return coarse_apply(C, o, v, nrhs, prec, stream); };
  auto norms = [&](const float2* v, int dst, int mode) -> int {
    c->launches += 2;
    k_mnorm<<<gr, MT, 0, st>>>(v, rows, nrhs, pt);
    k_mscalars<<<1, 64, 0, st>>>(pt, gr, nrhs, sc, dst, mode);
    DWF_CUDA(c, cudaGetLastError());
    return DWF_OK;
  };
  // b = A rhs; r = b; p = r; e = 0; rr = |b|^2 per rhs
  DWF_CUDA(c, cudaMemsetAsync(sc, 0, 5 * 64 * sizeof(double), st));
  DWF_CUDA(c, cudaMemsetAsync(e, 0, n * sizeof(float2), st));
  if ((rc = apply(r, (const float2*)rhs))) return rc;
  DWF_CUDA(c, cudaMemcpyAsync(p, r, n * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  if ((rc = norms(r, 0, 0))) return rc;
  std::vector<double> h(5 * 64), bb(nrhs);
  DWF_CUDA(c, cudaMemcpyAsync(h.data(), sc, 5 * 64 * sizeof(double), cudaMemcpyDeviceToHost, st));
  DWF_CUDA(c, cudaStreamSynchronize(st));
  for (int k = 0; k < nrhs; k++) {
    bb[k] = h[5 * k];
    if (!isfinite(bb[k])) return dwf_fail(c, DWF_ENAN, "coarse_solve_multi: source is not finite");
    if (iters) iters[k] = 0;
  }
  std::vector<double> done(nrhs, 0.0);
  for (int k = 0; k < nrhs; k++)
    if (!(bb[k] > 0)) done[k] = 1.0;
  auto push_done = [&]() -> int {
    for (int k = 0; k < nrhs; k++) h[5 * k + 4] = done[k];
    for (int k = 0; k < nrhs; k++)
      DWF_CUDA(c, cudaMemcpyAsync(sc + 5 * k + 4, &h[5 * k + 4], sizeof(double), cudaMemcpyHostToDevice, st));
    return DWF_OK;
  };
  if ((rc = push_done())) return rc;
  int it = 0, active = 0;
  for (int k = 0; k < nrhs; k++) active += done[k] == 0.0;
  while (active > 0 && it < maxiter) {
    // t = A p, q = A t; alpha = rr / |t|^2; e += alpha p; r -= alpha q;
    // beta = |r|^2 / rr; p = r + beta p
    if ((rc = apply(t, p))) return rc;
    if ((rc = norms(t, 1, 1))) return rc;
    if ((rc = apply(q, t))) return rc;
    c->launches++;
    k_mupdate<<<g, MT, 0, st>>>((float2*)e, r, p, q, n, nrhs, sc);
    if ((rc = norms(r, 1, 2))) return rc;
    c->launches++;
    k_mdir<<<g, MT, 0, st>>>(p, r, n, nrhs, sc);
    DWF_CUDA(c, cudaGetLastError());
    it++;
    if (it % 8 == 0 || it == maxiter) {
      DWF_CUDA(c, cudaMemcpyAsync(h.data(), sc, 5 * 64 * sizeof(double), cudaMemcpyDeviceToHost, st));
      DWF_CUDA(c, cudaStreamSynchronize(st));
      bool changed = false;
      for (int k = 0; k < nrhs; k++) {
        if (done[k] != 0.0) continue;
        if (!isfinite(h[5 * k])) return dwf_fail(c, DWF_ENAN, "coarse_solve_multi: NaN");
        if (h[5 * k] <= tol * tol * bb[k]) {
          done[k] = 1.0;
          if (iters) iters[k] = it;
          changed = true;
        }
      }
      if (changed) {
        if ((rc = push_done())) return rc;
        active = 0;
        for (int k = 0; k < nrhs; k++) active += done[k] == 0.0;
      }
    }
  }
  for (int k = 0; k < nrhs; k++)
    if (done[k] == 0.0 && iters) iters[k] = it;
  DWF_CUDA(c, cudaStreamSynchronize(st));
  if (prec == DWF_TF32) {
    rc = coarse_apply_status(C, stream);
    if (rc) return rc;
  }
  return active > 0 ? dwf_fail(c, DWF_ENOCONV, "coarse_solve_multi: maxiter reached before tol") : DWF_OK;
}
