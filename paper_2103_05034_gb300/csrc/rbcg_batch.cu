// Batched red-black CGNR: nrhs independent systems, each with its own quark
// mass, solved together (Sec. 5.1 operator; the HMC setting of Sec. 6, where
// several pseudofermions with Hasenbusch masses are solved on one gauge
// field).  Every CG iteration is one set of hopping launches over all systems
// still iterating (grid.y = system), so the links are read once per launch for
// the batch, and the M5 / mf term and M_ee^-1 of each system use its own mass.
// Each system runs its own CG recurrence (its scalars rr, pAp, alpha, beta
// live in its bank of the device scalars; alpha enters the fused update
// epilogue of the hopping kernel per system, beta the batched p update) and
// takes its own FP64 reliable updates, exactly when the single-system solver
// would.  A system whose FP64 true residual reaches tol leaves the batch: its
// vectors are swapped behind the active ones, so the launches shrink to the
// systems still iterating.
#include <chrono>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#include "dwf_internal.cuh"

namespace {

int bank(int i, int k) { return S_BANK0 + i * S_BANK + k; }

HopLaunch hop(void* out, const void* in, int po, int dag, int nrhs, double alpha) {
  HopLaunch h;
  memset(&h, 0, sizeof(h));
  h.out = out;
  h.in = in;
  h.out_parity = po;
  h.dagger = dag;
  h.nrhs = nrhs;
  h.alpha = alpha;
  return h;
}

// Per-system vectors, nrhs consecutive even half fields each.  rhs and bp are
// permuted with the systems, so they are solver-owned copies.
struct BatchBufs {
  void* rhs;  // M_pc^dag b'_e (red-black) or phi (normal equations), FP64
  void* bp;   // b'_e (red-black) or null
  void *rhi, *yhi, *ohi, *xlo, *rlo, *p, *Ap, *ylo, *olo;
};

// Per-system |v_i|^2 of n consecutive half fields into bank slot k.
int norms(dwf_ctx* c, const void* v, int prec, int n, int64_t he, int k, cudaStream_t st) {
  const size_t stride = (size_t)he * dwf_complex_bytes(prec);
  for (int i = 0; i < n; i++) {
    int rc = norm2_dev(c, (const char*)v + i * stride, he, prec, bank(i, k), st);
    if (rc) return rc;
  }
  return DWF_OK;
}

// CG on M_pc(m_i)^dag M_pc(m_i) x_i = rhs_i for i < n.  x_e: n FP64 even
// fields (output, in the input order); bnorm[i] > 0 is the norm the residual
// of system i is measured against; mm[i] accumulates its half-lattice
// hopping terms.
int cg_core_batch(dwf_ctx* c, double2* x_e, const BatchBufs& B, const double* bnorm_in, int n, double tol,
                  int maxiter, int plo, const double* mf_in, dwf_solve_stats* S, std::vector<double>& mm,
                  cudaStream_t st) {
  const int64_t he = c->g.Vh * 12 * c->g.Ls;
  const int64_t hn = he * n;
  const size_t cb = dwf_complex_bytes(plo), h64 = he * 16, hlo = he * cb;
  int rc;
  DWF_CUDA(c, cudaMemsetAsync(x_e, 0, hn * 16, st));
  if (plo != DWF_F64) DWF_CUDA(c, cudaMemsetAsync(B.xlo, 0, hn * cb, st));
  void* xin = plo == DWF_F64 ? (void*)x_e : B.xlo;
  const double delta = 0.1;
  // host state per slot; slot k holds system sys[k]; slots < na iterate
  std::vector<int> sys(n);
  std::vector<double> mass(mf_in, mf_in + n), bnorm(bnorm_in, bnorm_in + n);
  std::vector<double> true_res(n, 0.0), rho(n, 1.0), rr_max(n, 0.0), rr_last(n, 0.0);
  std::vector<char> have_x(n, 0), restart_p(n, 0);
  std::vector<int> iters(n, 0), updates(n, 0);
  for (int i = 0; i < n; i++) sys[i] = i;
  int na = n, it = 0;
  auto v64 = [&](void* base, int k) { return (void*)((char*)base + k * h64); };
  auto vlo = [&](void* base, int k) { return (void*)((char*)base + k * hlo); };

  // FP64 reliable update of slot k, as in the single-system solver: fold the
  // inner x into x (FP64), recompute the true residual, restart rr.
  auto reliable = [&](int k) -> int {
    int r;
    const double* m = &mass[k];
    void *xk = v64(x_e, k), *rh = v64(B.rhi, k), *yh = v64(B.yhi, k), *oh = v64(B.ohi, k);
    void *rl = vlo(B.rlo, k), *yl = vlo(B.ylo, k), *ol = vlo(B.olo, k);
    const void* rhs = v64(B.rhs, k);
    const void* bp = B.bp ? v64(B.bp, k) : nullptr;
    if (plo != DWF_F64) {
      void* xl = vlo(B.xlo, k);
      if (have_x[k]) {
        r = blas_axpby(c, 1.0, xl, plo, 1.0, xk, DWF_F64, he, st);
        if (r) return r;
      }
      DWF_CUDA(c, cudaMemsetAsync(xl, 0, hlo, st));
    }
    if (have_x[k]) {
      // FP32 operator on x rounded to FP32 while the residual is far above
      // FP32 rounding, FP64 otherwise (as in the single-system solve)
      if (plo == DWF_F32 && bp && true_res[k] > 1e-4) {
        void* al = vlo(B.Ap, k);
        r = blas_copy(c, yl, DWF_F32, xk, DWF_F64, he, st);
        if (r) return r;
        r = mpc_apply(c, al, yl, ol, m, 0, DWF_F32, 1, 0, st, nullptr);
        if (r) return r;
        r = blas_copy(c, yh, DWF_F64, al, DWF_F32, he, st);
      } else {
        r = mpc_apply(c, yh, xk, oh, m, 0, DWF_F64, 1, 0, st, nullptr);
      }
      if (r) return r;
      if (bp) {  // y = b'_e - M_pc x (true residual), r = M_pc^dag y
        r = blas_axpby(c, 1.0, bp, DWF_F64, -1.0, yh, DWF_F64, he, st);
        if (r) return r;
        r = norm2_dev(c, yh, he, DWF_F64, bank(k, S_BT0), st);
        if (r) return r;
        if (plo == DWF_F64) {
          r = mpc_apply(c, rh, yh, oh, m, 1, DWF_F64, 1, 0, st, nullptr);
        } else {
          r = blas_copy(c, yl, plo, yh, DWF_F64, he, st);
          if (r) return r;
          r = mpc_apply(c, rl, yl, ol, m, 1, plo, 1, 0, st, nullptr);
          if (r) return r;
          r = blas_copy(c, rh, DWF_F64, rl, plo, he, st);
        }
      } else {  // r = rhs - M^dag M x
        r = mpc_apply(c, rh, yh, oh, m, 1, DWF_F64, 1, 0, st, nullptr);
        if (r) return r;
        r = blas_axpby(c, 1.0, rhs, DWF_F64, -1.0, rh, DWF_F64, he, st);
        if (r) return r;
        r = norm2_dev(c, rh, he, DWF_F64, bank(k, S_BT0), st);
      }
      if (r) return r;
      mm[sys[k]] += 4;
      updates[sys[k]]++;
    } else {
      r = blas_copy(c, rh, DWF_F64, rhs, DWF_F64, he, st);
      if (r) return r;
      r = norm2_dev(c, bp ? bp : rhs, he, DWF_F64, bank(k, S_BT0), st);
      if (r) return r;
    }
    r = norm2_dev(c, rh, he, DWF_F64, bank(k, S_BT1), st);
    if (r) return r;
    r = blas_copy(c, rl, plo, rh, DWF_F64, he, st);
    if (r) return r;
    r = norm2_dev(c, rl, he, plo, bank(k, S_RR), st);
    if (r) return r;
    // restore <r, p> = |r|^2 for the kept direction (see the single-system
    // solver), or restart it when the recurrence was diverging
    void* pk = vlo(B.p, k);
    const bool had_x = have_x[k], fix_p = had_x && !restart_p[k];
    if (fix_p) {
      int np = 0;
      r = blas_cdot_partials(c, rl, pk, he, plo, st, &np);
      if (r) return r;
      r = blas_finalize(c, np, 2, bank(k, S_BDOT), st);
      if (r) return r;
    }
    r = read_scalars(c, bank(k, 0), S_BANK, st);
    if (r) return r;
    const double* q = c->hscal + bank(k, 0);
    if (fix_p && q[S_RR] > 0) {
      r = blas_caxpy(c, 1.0 - q[S_BDOT] / q[S_RR], -q[S_BDOT + 1] / q[S_RR], rl, plo, pk, plo, he, st);
      if (r) return r;
    } else if (had_x) {
      r = blas_copy(c, pk, plo, rl, plo, he, st);
      if (r) return r;
    }
    restart_p[k] = 0;
    true_res[k] = sqrt(q[S_BT0]) / bnorm[k];
    const double rr_hi = q[S_BT1];
    if (!std::isfinite(true_res[k]) || !std::isfinite(rr_hi)) return dwf_fail(c, DWF_ENAN, "NaN in CG residual");
    rho[k] = rr_hi > 0 ? sqrt(q[S_BT0] / rr_hi) : 1.0;
    rr_max[k] = rr_hi;
    rr_last[k] = rr_hi;
    have_x[k] = 1;
    return DWF_OK;
  };

  // exchange slots a and b: vectors, device scalars and host state
  auto swap_slots = [&](int a, int b) -> int {
    if (a == b) return DWF_OK;
    int r = blas_swap(c, v64(x_e, a), v64(x_e, b), h64, st);
    if (!r) r = blas_swap(c, v64(B.rhs, a), v64(B.rhs, b), h64, st);
    if (!r && B.bp) r = blas_swap(c, v64(B.bp, a), v64(B.bp, b), h64, st);
    if (!r && plo != DWF_F64) r = blas_swap(c, vlo(B.xlo, a), vlo(B.xlo, b), hlo, st);
    if (!r) r = blas_swap(c, vlo(B.rlo, a), vlo(B.rlo, b), hlo, st);
    if (!r) r = blas_swap(c, vlo(B.p, a), vlo(B.p, b), hlo, st);
    if (!r) r = blas_swap(c, c->dscal + bank(a, 0), c->dscal + bank(b, 0), S_BANK * sizeof(double), st);
    if (r) return r;
    std::swap(sys[a], sys[b]);
    std::swap(mass[a], mass[b]);
    std::swap(bnorm[a], bnorm[b]);
    std::swap(true_res[a], true_res[b]);
    std::swap(rho[a], rho[b]);
    std::swap(rr_max[a], rr_max[b]);
    std::swap(rr_last[a], rr_last[b]);
    std::swap(have_x[a], have_x[b]);
    std::swap(restart_p[a], restart_p[b]);
    return DWF_OK;
  };
  // converged systems leave the active range [0, na)
  auto compact = [&]() -> int {
    for (int k = na - 1; k >= 0; k--) {
      if (true_res[k] > tol) continue;
      iters[sys[k]] = it;
      int r = swap_slots(k, na - 1);
      if (r) return r;
      na--;
    }
    return DWF_OK;
  };

  for (int k = 0; k < n; k++) {
    rc = reliable(k);
    if (rc) return rc;
  }
  rc = blas_copy(c, B.p, plo, B.rlo, plo, hn, st);
  if (rc) return rc;
  rc = compact();
  if (rc) return rc;
  const int check_every = 8;
  std::vector<double> mview(n);
  while (na > 0 && it < maxiter) {
    for (int k = 0; k < na; k++) mview[k] = mass[k];
    // y = M_pc p with |y_k|^2 = <p_k, A_k p_k> -> alpha_k
    int np = 0;
    rc = mpc_apply(c, B.ylo, B.p, B.olo, mview.data(), 0, plo, na, 1, st, &np);
    if (rc) return rc;
    rc = blas_finalize_batch(c, np / na, na, S_PAP, 1, st);
    if (rc) return rc;
    // A p = M_pc^dag y, whose second hopping launch updates x_k += alpha_k p_k,
    // r_k -= alpha_k A p_k and reduces |r_k|^2
    HopLaunch h1 = hop(B.olo, B.ylo, 1, 1, na, -0.5);
    h1.inv_mode = 2;
    h1.mf = mview.data();
    rc = launch_hop(c, h1, plo, st, nullptr);
    if (rc) return rc;
    HopLaunch h2 = hop(nullptr, B.olo, 0, 1, na, 0.5);
    h2.aux = B.ylo;
    h2.aux_mode = 3;
    h2.mf = mview.data();
    h2.reduce = 1;
    h2.cg_x = xin;
    h2.cg_r = B.rlo;
    h2.cg_p = B.p;
    h2.cg_alpha = c->dscal + bank(0, S_ALPHA);
    h2.cg_alpha_stride = S_BANK;
    rc = launch_hop(c, h2, plo, st, &np);
    if (rc) return rc;
    rc = blas_finalize_batch(c, np / na, na, S_RRNEW, 2, st);
    if (rc) return rc;
    rc = blas_cg_p_batch(c, B.p, B.rlo, he, na, plo, st);
    if (rc) return rc;
    for (int k = 0; k < na; k++) mm[sys[k]] += 4;
    it++;
    if (it % check_every == 0 || it == maxiter) {
      rc = read_scalars(c, S_BANK0, na * S_BANK, st);
      if (rc) return rc;
      std::vector<int> fire;
      for (int k = 0; k < na; k++) {
        const double rr_lo = c->hscal[bank(k, S_RR)];
        if (!std::isfinite(rr_lo)) return dwf_fail(c, DWF_ENAN, "NaN in CG residual");
        if (rr_lo > rr_max[k]) rr_max[k] = rr_lo;
        const bool diverging = rr_lo > 1e4 * rr_last[k];
        if (diverging) restart_p[k] = 1;
        if (rr_lo < delta * delta * rr_max[k] || rho[k] * sqrt(rr_lo) / bnorm[k] <= tol || it == maxiter ||
            diverging)
          fire.push_back(k);
      }
      for (int k : fire) {
        rc = reliable(k);
        if (rc) return rc;
      }
      if (!fire.empty()) {
        rc = compact();
        if (rc) return rc;
      }
    }
  }
  for (int k = 0; k < na; k++) iters[sys[k]] = it;
  // x back into the input order (yhi as the staging buffer)
  for (int k = 0; k < n; k++)
    DWF_CUDA(c, cudaMemcpyAsync(v64(B.yhi, sys[k]), v64(x_e, k), h64, cudaMemcpyDeviceToDevice, st));
  DWF_CUDA(c, cudaMemcpyAsync(x_e, B.yhi, hn * 16, cudaMemcpyDeviceToDevice, st));
  for (int k = 0; k < n; k++) {
    const int i = sys[k];
    S[i].iterations = iters[i];
    S[i].true_residual = true_res[k];
    S[i].reliable_updates = updates[i];
  }
  return DWF_OK;
}

int check_batch(dwf_ctx* c, const void* x, const void* b, const double* mf, int nrhs, double tol,
                int maxiter) {
  if (!c) return DWF_EINVAL;
  if (!x || !b || !mf) return dwf_fail(c, DWF_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > DWF_MAX_RHS) return dwf_fail(c, DWF_EINVAL, "nrhs out of range");
  if (!(tol > 0) || maxiter < 1) return dwf_fail(c, DWF_EINVAL, "bad tol or maxiter");
  for (int i = 0; i < nrhs; i++)
    if (!std::isfinite(mf[i])) return dwf_fail(c, DWF_EINVAL, "mass is not finite");
  return DWF_OK;
}

double now_sec() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// FP64 norms of nrhs sources given as parity halves; zero sources get
// bnorm = 1 (their solution is zero and their residual ratio zero).
int source_norms(dwf_ctx* c, const void* be, const void* bo, int n, int64_t he, std::vector<double>& bnorm,
                 std::vector<char>& zero, cudaStream_t st) {
  int rc = norms(c, be, DWF_F64, n, he, S_BT0, st);
  if (rc) return rc;
  if (bo) {
    rc = norms(c, bo, DWF_F64, n, he, S_BT1, st);
    if (rc) return rc;
  }
  rc = read_scalars(c, S_BANK0, n * S_BANK, st);
  if (rc) return rc;
  bnorm.assign(n, 1.0);
  zero.assign(n, 0);
  for (int i = 0; i < n; i++) {
    const double* q = c->hscal + bank(i, 0);
    const double b2 = q[S_BT0] + (bo ? q[S_BT1] : 0.0);
    if (!std::isfinite(b2)) return dwf_fail(c, DWF_ENAN, "source is not finite");
    if (b2 > 0)
      bnorm[i] = sqrt(b2);
    else
      zero[i] = 1;
  }
  return DWF_OK;
}

}  // namespace

extern "C" int rbcg_solve_batch(dwf_ctx* c, void* x, const void* b, const double* mf, int nrhs, double tol,
                                int maxiter, int policy, dwf_solve_stats* stats, void* stream) {
  const double t0 = now_sec();
  int rc = check_batch(c, x, b, mf, nrhs, tol, maxiter);
  if (rc) return rc;
  if (policy != DWF_SOLVE_F64 && policy != DWF_SOLVE_MIXED_F32) return dwf_fail(c, DWF_EINVAL, "bad policy");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = nrhs;
  const int plo = policy == DWF_SOLVE_F64 ? DWF_F64 : DWF_F32;
  const int64_t he = c->g.Vh * 12 * c->g.Ls, hn = he * n;
  const size_t b64 = hn * 16, blo = hn * dwf_complex_bytes(plo), h16 = he * 16;
  const bool host_b = !dwf_is_device_ptr(b), host_x = !dwf_is_device_ptr(x);
  if (host_b != host_x) return dwf_fail(c, DWF_EINVAL, "x and b must be both host or both device");
  if (!host_b && (((uintptr_t)b & 15) || ((uintptr_t)x & 15))) return dwf_fail(c, DWF_EINVAL, "alignment");
  double2* be = (double2*)dwf_workspace(c, WS_BE, b64);
  double2* bo = (double2*)dwf_workspace(c, WS_BO, b64);
  double2* xe = (double2*)dwf_workspace(c, WS_XE, b64);
  double2* xo = (double2*)dwf_workspace(c, WS_XO, b64);
  BatchBufs B;
  void* bp = dwf_workspace(c, WS_BP, b64);
  void* rhs = dwf_workspace(c, WS_RHS, b64);
  B.rhs = rhs;
  B.bp = bp;
  B.rhi = dwf_workspace(c, WS_RHI, b64);
  B.yhi = dwf_workspace(c, WS_YHI, b64);
  B.ohi = dwf_workspace(c, WS_OHI, b64);
  B.xlo = plo == DWF_F64 ? nullptr : dwf_workspace(c, WS_XLO, blo);
  B.rlo = dwf_workspace(c, WS_RLO, blo);
  B.p = dwf_workspace(c, WS_P, blo);
  B.Ap = dwf_workspace(c, WS_AP, blo);
  B.ylo = dwf_workspace(c, WS_YLO, blo);
  B.olo = dwf_workspace(c, WS_OLO, blo);
  char* full = (char*)dwf_workspace(c, WS_FULL, 2 * b64);
  if (!be || !bo || !xe || !xo || !bp || !rhs || !B.rhi || !B.yhi || !B.ohi || (plo != DWF_F64 && !B.xlo) ||
      !B.rlo || !B.p || !B.Ap || !B.ylo || !B.olo || !full)
    return dwf_fail(c, DWF_ENOMEM, "solver workspace");
  // split the full sources [rhs][even, odd] into parity-major batches
  const cudaMemcpyKind kin = host_b ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  for (int i = 0; i < n; i++) {
    const char* bi = (const char*)b + 2 * i * h16;
    DWF_CUDA(c, cudaMemcpyAsync((char*)be + i * h16, bi, h16, kin, st));
    DWF_CUDA(c, cudaMemcpyAsync((char*)bo + i * h16, bi + h16, h16, kin, st));
  }
  std::vector<double> bnorm;
  std::vector<char> zero;
  rc = source_norms(c, be, bo, n, he, bnorm, zero, st);
  if (rc) return rc;
  // b'_e = b_e + 1/2 D_eo M_oo^-1 b_o;  rhs = M_pc^dag b'_e
  rc = launch_mooee(c, B.ohi, bo, mf, 0, 1, DWF_F64, n, 0, st);
  if (rc) return rc;
  {
    HopLaunch h = hop(bp, B.ohi, 0, 0, n, 0.5);
    h.aux = be;
    h.aux_mode = 1;
    rc = launch_hop(c, h, DWF_F64, st, nullptr);
    if (rc) return rc;
  }
  rc = mpc_apply(c, rhs, bp, B.ohi, mf, 1, DWF_F64, n, 0, st, nullptr);
  if (rc) return rc;
  std::vector<double> mm(n, 3.0);  // half-lattice hopping terms per system
  std::vector<dwf_solve_stats> S(n);
  memset(S.data(), 0, n * sizeof(dwf_solve_stats));
  rc = cg_core_batch(c, xe, B, bnorm.data(), n, tol, maxiter, plo, mf, S.data(), mm, st);
  if (rc) return rc;
  // x_o = M_oo^-1 (b_o + 1/2 D_oe x_e)
  {
    HopLaunch h = hop(xo, xe, 1, 0, n, 0.5);
    h.aux = bo;
    h.aux_mode = 1;
    h.inv_mode = 1;
    h.mf = mf;
    rc = launch_hop(c, h, DWF_F64, st, nullptr);
    if (rc) return rc;
  }
  // true residuals ||b - D_DW x|| / ||b|| in FP64, parity by parity:
  // (D_DW x)_p = M x_p - 1/2 D_hop x_{1-p}
  char* fe = full;
  char* fo = full + b64;
  for (int po = 0; po < 2; po++) {
    HopLaunch h = hop(po ? fo : fe, po ? (const void*)xe : (const void*)xo, po, 0, n, -0.5);
    h.aux = po ? (const void*)xo : (const void*)xe;
    h.aux_mode = 2;
    h.mf = mf;
    rc = launch_hop(c, h, DWF_F64, st, nullptr);
    if (rc) return rc;
    rc = blas_axpby(c, 1.0, po ? (const void*)bo : (const void*)be, DWF_F64, -1.0, po ? fo : fe, DWF_F64, hn,
                    st);
    if (rc) return rc;
  }
  rc = norms(c, fe, DWF_F64, n, he, S_BT0, st);
  if (rc) return rc;
  rc = norms(c, fo, DWF_F64, n, he, S_BT1, st);
  if (rc) return rc;
  // the solutions back into the caller's [rhs][even, odd] layout
  const cudaMemcpyKind kout = host_x ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  for (int i = 0; i < n; i++) {
    char* xi = (char*)x + 2 * i * h16;
    DWF_CUDA(c, cudaMemcpyAsync(xi, (const char*)xe + i * h16, h16, kout, st));
    DWF_CUDA(c, cudaMemcpyAsync(xi + h16, (const char*)xo + i * h16, h16, kout, st));
  }
  rc = read_scalars(c, S_BANK0, n * S_BANK, st);
  if (rc) return rc;
  bool ok = true;
  const double sec = now_sec() - t0;
  for (int i = 0; i < n; i++) {
    const double* q = c->hscal + bank(i, 0);
    S[i].true_residual = zero[i] ? 0.0 : sqrt(q[S_BT0] + q[S_BT1]) / bnorm[i];
    S[i].fine_matmuls = (mm[i] + 3.0) / 2.0;  // + reconstruction and residual
    S[i].seconds = sec;
    S[i].status = S[i].true_residual <= tol ? DWF_OK : DWF_ENOCONV;
    if (S[i].status) ok = false;
    if (stats) stats[i] = S[i];
  }
  DWF_CUDA(c, cudaGetLastError());
  if (!ok) return dwf_fail(c, DWF_ENOCONV, "maxiter reached before tol");
  return DWF_OK;
}

extern "C" int rbcg_normal_solve_batch(dwf_ctx* c, void* x, const void* phi, const double* mf, int nrhs,
                                       double tol, int maxiter, int policy, dwf_solve_stats* stats,
                                       void* stream) {
  const double t0 = now_sec();
  int rc = check_batch(c, x, phi, mf, nrhs, tol, maxiter);
  if (rc) return rc;
  if (policy != DWF_SOLVE_F64 && policy != DWF_SOLVE_MIXED_F32) return dwf_fail(c, DWF_EINVAL, "bad policy");
  if (!dwf_is_device_ptr(x) || !dwf_is_device_ptr(phi)) return dwf_fail(c, DWF_EINVAL, "device buffers required");
  if (((uintptr_t)x & 15) || ((uintptr_t)phi & 15)) return dwf_fail(c, DWF_EINVAL, "alignment");
  if (x == phi) return dwf_fail(c, DWF_EINVAL, "x must not alias phi");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = nrhs;
  const int plo = policy == DWF_SOLVE_F64 ? DWF_F64 : DWF_F32;
  const int64_t he = c->g.Vh * 12 * c->g.Ls, hn = he * n;
  const size_t b64 = hn * 16, blo = hn * dwf_complex_bytes(plo);
  BatchBufs B;
  B.rhs = dwf_workspace(c, WS_RHS, b64);  // permuted with the systems: a copy
  B.bp = nullptr;
  B.rhi = dwf_workspace(c, WS_RHI, b64);
  B.yhi = dwf_workspace(c, WS_YHI, b64);
  B.ohi = dwf_workspace(c, WS_OHI, b64);
  B.xlo = plo == DWF_F64 ? nullptr : dwf_workspace(c, WS_XLO, blo);
  B.rlo = dwf_workspace(c, WS_RLO, blo);
  B.p = dwf_workspace(c, WS_P, blo);
  B.Ap = dwf_workspace(c, WS_AP, blo);
  B.ylo = dwf_workspace(c, WS_YLO, blo);
  B.olo = dwf_workspace(c, WS_OLO, blo);
  if (!B.rhs || !B.rhi || !B.yhi || !B.ohi || (plo != DWF_F64 && !B.xlo) || !B.rlo || !B.p || !B.Ap ||
      !B.ylo || !B.olo)
    return dwf_fail(c, DWF_ENOMEM, "solver workspace");
  DWF_CUDA(c, cudaMemcpyAsync(B.rhs, phi, b64, cudaMemcpyDeviceToDevice, st));
  std::vector<double> bnorm;
  std::vector<char> zero;
  rc = source_norms(c, phi, nullptr, n, he, bnorm, zero, st);
  if (rc) return rc;
  std::vector<dwf_solve_stats> S(n);
  memset(S.data(), 0, n * sizeof(dwf_solve_stats));
  std::vector<double> mm(n, 0.0);
  rc = cg_core_batch(c, (double2*)x, B, bnorm.data(), n, tol, maxiter, plo, mf, S.data(), mm, st);
  if (rc) return rc;
  DWF_CUDA(c, cudaStreamSynchronize(st));
  bool ok = true;
  const double sec = now_sec() - t0;
  for (int i = 0; i < n; i++) {
    S[i].fine_matmuls = mm[i] / 2.0;
    S[i].seconds = sec;
    S[i].status = S[i].true_residual <= tol ? DWF_OK : DWF_ENOCONV;
    if (S[i].status) ok = false;
    if (stats) stats[i] = S[i];
  }
  DWF_CUDA(c, cudaGetLastError());
  if (!ok) return dwf_fail(c, DWF_ENOCONV, "maxiter reached before tol");
  return DWF_OK;
}
