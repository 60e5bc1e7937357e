// Pseudofermion force for HMC with the red-black operator of Sec. 5.1 of
// arXiv:2103.05034 (the paper places its solvers inside HMC, Sec. 6; the force
// is derived from first principles).  For S = phi^dag (M^dag M)^-1 phi,
// M = M_pc, X = (M^dag M)^-1 phi (even), Y = M X, and the full fields
// X' = X + M_oo^-1 M_oe X, Y' = Y + M_oo^-dag M_eo^dag Y:
//   G_mu(x) = TA(U_mu(x) A_mu(x) - B_mu(x) U_mu(x)^dag),
//   A_mu(x)_ab = sum_s Y'_s(x)^dag_b (1 - gamma_mu) X'_s(x+mu)_a,
//   B_mu(x)_ab = sum_s Y'_s(x+mu)^dag_b (1 + gamma_mu) X'_s(x)_a,
// so that dS/deps = sum Re tr(G^dag Q) for U -> exp(eps Q) U, Q in su(3).
// Each spin trace is a two-spinor product: Y^dag (1 -+ gamma) X = h_Y^dag h_X
// with both fields projected by the same (1 -+ gamma) half-spinor map.
#include <math.h>
#include <string.h>

#include <type_traits>
#include <vector>

#include "dhop_impl.cuh"
#include "dwf_internal.cuh"

namespace {

template <class R, int MU>
__device__ __forceinline__ void proj(cpx<R> (&h)[2][3], const cpx<R> (&ps)[12], R sg) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const cpx<R> p0 = ps[c], p1 = ps[3 + c], p2 = ps[6 + c], p3 = ps[9 + c];
    if (MU == 0) {
      h[0][c] = cmake<R>(p0.re - sg * p3.im, p0.im + sg * p3.re);
      h[1][c] = cmake<R>(p1.re - sg * p2.im, p1.im + sg * p2.re);
    } else if (MU == 1) {
      h[0][c] = cmake<R>(p0.re + sg * p3.re, p0.im + sg * p3.im);
      h[1][c] = cmake<R>(p1.re - sg * p2.re, p1.im - sg * p2.im);
    } else if (MU == 2) {
      h[0][c] = cmake<R>(p0.re - sg * p2.im, p0.im + sg * p2.re);
      h[1][c] = cmake<R>(p1.re + sg * p3.im, p1.im - sg * p3.re);
    } else {
      h[0][c] = cmake<R>(p0.re - sg * p2.re, p0.im - sg * p2.im);
      h[1][c] = cmake<R>(p1.re - sg * p3.re, p1.im - sg * p3.im);
    }
  }
}

// o_ab = sum_k hx[k][a] conj(hy[k][b]) (one s-slice)
template <class R>
__device__ __forceinline__ void outer2(cpx<R> (&o)[9], const cpx<R> (&hx)[2][3], const cpx<R> (&hy)[2][3]) {
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      R re = 0, im = 0;
#pragma unroll
      for (int k = 0; k < 2; k++) {
        re += hx[k][a].re * hy[k][b].re + hx[k][a].im * hy[k][b].im;
        im += hx[k][a].im * hy[k][b].re - hx[k][a].re * hy[k][b].im;
      }
      o[a * 3 + b] = cmake<R>(re, im);
    }
}

// Sum over the Ls threads of each site of one 3x3 complex matrix per thread
// (shared-memory reduction, fixed order), added to AB[site][slot] in FP64.
template <class R, int LS, int SB>
__device__ __forceinline__ void site_sum(R* red, double2* AB, int slot, const cpx<R> (&o)[9], int sl, int s,
                                         double coef) {
  constexpr int NT = LS * SB;
#pragma unroll
  for (int e = 0; e < 9; e++) {
    red[((sl * LS + s) * 9 + e) * 2] = o[e].re;
    red[((sl * LS + s) * 9 + e) * 2 + 1] = o[e].im;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < SB * 18; t += NT) {
    const int sl2 = t / 18, e = t - sl2 * 18;
    R acc = 0;
    for (int q = 0; q < LS; q++) acc += red[(sl2 * LS + q) * 18 + e];
    double* dst = (double*)(AB + (sl2 * 8 + slot) * 9);
    dst[e] += coef * (double)acc;
  }
  __syncthreads();
}

// Weight of each field pair in the sum (+1 for a pseudofermion; +1 and -1
// for the two bilinears of a Hasenbusch ratio factor).
struct ForceCoef {
  double c[DWF_MAX_RHS];
};

// One CTA: SB checkerboard sites of one parity x Ls threads (s fastest, so
// the neighbours' spinors are read as contiguous Ls-runs), all npf
// pseudofermions (field pairs f, each weighted by coef.c[f]).  Each thread forms the s-slice of A_mu and B_mu for the 4
// directions; the Ls slices (and the pseudofermions, G being linear in A and
// B) are summed per site in shared memory, and 4 threads per site form G_mu,
// reading each link once for all pseudofermions.  The final products run in
// the fields' precision (FP32 fields: FP32, FP64 fields: FP64), the sums and
// the force in FP64.
template <int P, int LS, int SB>
__global__ void __launch_bounds__(LS* SB) k_force(double2* force, const typename Prec<P>::S* Xe,
                                                 const typename Prec<P>::S* Xo, const typename Prec<P>::S* Ye,
                                                 const typename Prec<P>::S* Yo, long long fstride, int npf,
                                                 const typename Prec<P>::LS* links_e,
                                                 const typename Prec<P>::LS* links_o, int L0, int L1, int L2, int L3,
                                                 int Vh, const ForceCoef coef) {
  typedef typename Prec<P>::R R;
  typedef typename Prec<P>::S S;
  __shared__ R red[SB * LS * 18];
  __shared__ double2 AB[SB * 8 * 9];  // per site: A_mu (slots 0-3), B_mu (slots 4-7)
  const int tid = threadIdx.x, sl = tid / LS, s = tid - sl * LS;
  for (int i = tid; i < SB * 8 * 9; i += LS * SB) AB[i] = make_double2(0.0, 0.0);
  // (the first site_sum's barrier orders these stores before its additions)
  // the two parities of a block of sites are neighbouring CTAs, so that what
  // one reads as its own X, Y the other reads as neighbours while it is in L2
  // (parity-major order read every field twice from DRAM)
  const int p = blockIdx.x & 1;
  const int blk = blockIdx.x >> 1;
  const int h = blk * SB + sl;
  const bool active = h < Vh;
  const int hh = active ? h : 0;
  const int Lxh = L0 / 2;
  int rem = hh / Lxh;
  const int xh = hh - rem * Lxh;
  int x[4];
  x[1] = rem % L1;
  rem /= L1;
  x[2] = rem % L2;
  x[3] = rem / L2;
  x[0] = 2 * xh + ((x[1] + x[2] + x[3] + p) & 1);
  const int Ld[4] = {L0, L1, L2, L3};
  const long long row = 12LL * LS;
  // neighbour half-lattice indices in the +mu directions (other parity)
  int nbh[4];
#pragma unroll
  for (int mu = 0; mu < 4; mu++) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] = (y[mu] + 1 == Ld[mu]) ? 0 : y[mu] + 1;
    const long long ylex = y[0] + (long long)L0 * (y[1] + (long long)L1 * (y[2] + (long long)L2 * y[3]));
    nbh[mu] = (int)(ylex >> 1);
  }
  for (int f = 0; f < npf; f++) {
    const S* Xs = (p ? Xo : Xe) + f * fstride;  // fields of this site's parity
    const S* Ys = (p ? Yo : Ye) + f * fstride;
    const S* Xn = (p ? Xe : Xo) + f * fstride;  // and of the neighbours'
    const S* Yn = (p ? Ye : Yo) + f * fstride;
    cpx<R> xb[12], ya[12];
#pragma unroll
    for (int c = 0; c < 12; c++) {
      xb[c] = active ? ld_c(Xs + hh * row + c * LS + s) : cmake<R>(0, 0);
      ya[c] = active ? ld_c(Ys + hh * row + c * LS + s) : cmake<R>(0, 0);
    }
    auto dir = [&](auto muc) {
      constexpr int MU = decltype(muc)::value;
      const S* Xy = Xn + nbh[MU] * row + s;
      const S* Yy = Yn + nbh[MU] * row + s;
      cpx<R> xa[12], yb[12];
#pragma unroll
      for (int c = 0; c < 12; c++) {
        xa[c] = active ? ld_c(Xy + c * LS) : cmake<R>(0, 0);  // X'(x+mu)
        yb[c] = active ? ld_c(Yy + c * LS) : cmake<R>(0, 0);  // Y'(x+mu)
      }
      cpx<R> hx[2][3], hy[2][3], o[9];
      proj<R, MU>(hx, xa, R(1));
      proj<R, MU>(hy, ya, R(1));
      outer2<R>(o, hx, hy);
      site_sum<R, LS, SB>(red, AB, MU, o, sl, s, coef.c[f]);
      proj<R, MU>(hx, xb, R(-1));
      proj<R, MU>(hy, yb, R(-1));
      outer2<R>(o, hx, hy);
      site_sum<R, LS, SB>(red, AB, 4 + MU, o, sl, s, coef.c[f]);
    };
    dir(std::integral_constant<int, 0>());
    dir(std::integral_constant<int, 1>());
    dir(std::integral_constant<int, 2>());
    dir(std::integral_constant<int, 3>());
  }
  // G_mu = TA(U A - B U^dag), one thread per (site, mu)
  for (int t = tid; t < SB * 4; t += LS * SB) {
    const int sl2 = t >> 2, mu = t & 3;
    const int h2 = blk * SB + sl2;
    if (h2 >= Vh) continue;
    int r2 = h2 / Lxh;
    const int xh2 = h2 - r2 * Lxh;
    int z[4];
    z[1] = r2 % L1;
    r2 /= L1;
    z[2] = r2 % L2;
    z[3] = r2 / L2;
    z[0] = 2 * xh2 + ((z[1] + z[2] + z[3] + p) & 1);
    const long long zlex = z[0] + (long long)L0 * (z[1] + (long long)L1 * (z[2] + (long long)L2 * z[3]));
    const double2* A = AB + (sl2 * 8 + mu) * 9;
    const double2* B = AB + (sl2 * 8 + 4 + mu) * 9;
    const typename Prec<P>::LS* U = (p ? links_o : links_e) + ((long long)h2 * 8 + 2 * mu) * 9;
    cpx<R> Z[9];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) {
        R re = 0, im = 0;
#pragma unroll
        for (int k = 0; k < 3; k++) {
          const R ux = (R)U[a * 3 + k].x, uy = (R)U[a * 3 + k].y;  // (U A)_ab
          const R ax = (R)A[k * 3 + b].x, ay = (R)A[k * 3 + b].y;
          re += ux * ax - uy * ay;
          im += ux * ay + uy * ax;
          const R bx = (R)B[a * 3 + k].x, by = (R)B[a * 3 + k].y;  // (B U^dag)_ab = B_ak conj(U_bk)
          const R vx = (R)U[b * 3 + k].x, vy = (R)U[b * 3 + k].y;
          re -= bx * vx + by * vy;
          im -= by * vx - bx * vy;
        }
        Z[a * 3 + b] = cmake<R>(re, im);
      }
    // TA(Z) = (Z - Z^dag)/2 - tr(Z - Z^dag)/6
    const double trim = ((double)Z[0].im + (double)Z[4].im + (double)Z[8].im) / 3.0;  // i Im tr Z / 3
    double2* out = force + (zlex * 4 + mu) * 9;
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int b = 0; b < 3; b++) {
        double re = 0.5 * ((double)Z[a * 3 + b].re - (double)Z[b * 3 + a].re);
        double im = 0.5 * ((double)Z[a * 3 + b].im + (double)Z[b * 3 + a].im);
        if (a == b) im -= trim;
        out[a * 3 + b].x += re;
        out[a * 3 + b].y += im;
      }
  }
}

template <int P>
int launch_force(dwf_ctx* c, double2* force, const void* Xe, const void* Xo, const void* Ye, const void* Yo,
                 int npf, const ForceCoef& coef, cudaStream_t st) {
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::LS LT;
  const LT* le = P == DWF_F64 ? (const LT*)c->links64[0] : (const LT*)c->links32[0];
  const LT* lo = P == DWF_F64 ? (const LT*)c->links64[1] : (const LT*)c->links32[1];
  const long long fs = c->g.Vh * 12LL * c->g.Ls;
  c->launches++;
#define DWF_FORCE_CASE(LSV)                                                                                  \
  case LSV: {                                                                                                \
    constexpr int SB = LSV >= 16 ? 8 : 64 / LSV;                                                             \
    dim3 grid((unsigned)(2 * ((c->g.Vh + SB - 1) / SB)));                                                    \
    k_force<P, LSV, SB><<<grid, LSV * SB, 0, st>>>(force, (const S*)Xe, (const S*)Xo, (const S*)Ye,         \
                                                   (const S*)Yo, fs, npf, le, lo, c->g.L[0], c->g.L[1],      \
                                                   c->g.L[2], c->g.L[3], (int)c->g.Vh, coef);                \
    break;                                                                                                   \
  }
  switch (c->g.Ls) {
    DWF_FORCE_CASE(4)
    DWF_FORCE_CASE(8)
    DWF_FORCE_CASE(16)
    DWF_FORCE_CASE(24)
    default:
      return dwf_fail(c, DWF_EINVAL, "unsupported Ls");
  }
#undef DWF_FORCE_CASE
  return DWF_OK;
}

}  // namespace

// Odd halves of the field pairs and the force kernel: Xo (when not given) =
// M_oo^-1 M_oe Xe and Yo = M_oo^-dag M_eo^dag Ye, each pair f with its own
// mass mf[f]; then force += sum_f coef[f] G(X'_f, Y'_f).
static int force_tail(dwf_ctx* c, void* force, const void* Xe, void* Xo, bool have_xo, const void* Ye, void* Yo,
                      const double* mf, const ForceCoef& coef, int nf, int prec, cudaStream_t st) {
  int rc;
  if (!have_xo) {
    HopLaunch hx;
    memset(&hx, 0, sizeof(hx));
    hx.out = Xo;
    hx.in = Xe;
    hx.out_parity = 1;
    hx.nrhs = nf;
    hx.alpha = -0.5;
    hx.inv_mode = 1;
    hx.mf = mf;
    rc = launch_hop(c, hx, prec, st, nullptr);
    if (rc) return rc;
  }
  HopLaunch h;
  memset(&h, 0, sizeof(h));
  h.out = Yo;
  h.in = Ye;
  h.out_parity = 1;
  h.dagger = 1;
  h.nrhs = nf;
  h.alpha = -0.5;
  h.inv_mode = 2;
  h.mf = mf;
  rc = launch_hop(c, h, prec, st, nullptr);
  if (rc) return rc;
  rc = prec == DWF_F64 ? launch_force<DWF_F64>(c, (double2*)force, Xe, Xo, Ye, Yo, nf, coef, st)
                       : launch_force<DWF_F32>(c, (double2*)force, Xe, Xo, Ye, Yo, nf, coef, st);
  if (rc) return rc;
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}

static int force_args(dwf_ctx* c, const void* force, const void* X, int npf, int max_npf, int prec) {
  if (npf > max_npf) return dwf_fail(c, DWF_EINVAL, "npf out of range");
  if (prec != DWF_F64 && prec != DWF_F32) return dwf_fail(c, DWF_EINVAL, "bad precision");
  if (!dwf_is_device_ptr(force) || !dwf_is_device_ptr(X)) return dwf_fail(c, DWF_EINVAL, "device buffers required");
  if (((uintptr_t)force & 15) || ((uintptr_t)X & 15)) return dwf_fail(c, DWF_EINVAL, "alignment");
  return DWF_OK;
}

extern "C" int dwf_force(dwf_ctx* c, void* force, const void* X, const double* mf, int npf, int prec,
                         void* stream) {
  if (!c || !force || !X || !mf || npf < 1) return DWF_EINVAL;
  int rc = force_args(c, force, X, npf, DWF_MAX_RHS, prec);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t he = c->g.Vh * 12 * c->g.Ls;
  const size_t bytes = (size_t)npf * he * dwf_complex_bytes(prec);
  void* Xo = dwf_workspace(c, WS_FXO, bytes);
  void* Ye = dwf_workspace(c, WS_FYE, bytes);
  void* Yo = dwf_workspace(c, WS_FYO, bytes);
  if (!Xo || !Ye || !Yo) return dwf_fail(c, DWF_ENOMEM, "force workspace");
  // all pseudofermions at once, each with its own mass:
  // X_o = M_oo^-1 (-1/2 D_oe X_e) and Y_e = M_ee X_e + 1/2 D_eo X_o  (= M_pc X_e)
  rc = mpc_apply(c, Ye, X, Xo, mf, 0, prec, npf, 0, st, nullptr);
  if (rc) return rc;
  ForceCoef coef;
  for (int f = 0; f < DWF_MAX_RHS; f++) coef.c[f] = 1.0;
  return force_tail(c, force, X, Xo, true, Ye, Yo, mf, coef, npf, prec, st);
}

// Hasenbusch ratio factors S_r = phi^dag M2 (M1^dag M1)^-1 M2^dag phi: with
// X = (M1^dag M1)^-1 M2^dag phi, dS_r = 2 Re phi^dag dM2 X - 2 Re (M1 X)^dag
// dM1 X, so G_r = G(X', (M1 X)'; m1) - G(X', phi'; m2): two field pairs per
// factor in one force launch, weights +1 and -1.
extern "C" int dwf_ratio_force(dwf_ctx* c, void* force, const void* X, const void* phi, const double* m1,
                               const double* m2, int nratio, int prec, void* stream) {
  if (!c || !force || !X || !phi || !m1 || !m2 || nratio < 1) return DWF_EINVAL;
  int rc = force_args(c, force, X, nratio, DWF_MAX_RHS / 2, prec);
  if (rc) return rc;
  if (!dwf_is_device_ptr(phi) || ((uintptr_t)phi & 15)) return dwf_fail(c, DWF_EINVAL, "phi: aligned device buffer");
  for (int i = 0; i < nratio; i++)
    if (!isfinite(m1[i]) || !isfinite(m2[i])) return dwf_fail(c, DWF_EINVAL, "masses must be finite");
  cudaStream_t st = (cudaStream_t)stream;
  const int n = nratio;
  const int64_t he = c->g.Vh * 12 * c->g.Ls;
  const size_t fb = (size_t)he * dwf_complex_bytes(prec);
  void* Xe = dwf_workspace(c, WS_FXE, 2 * n * fb);
  void* Xo = dwf_workspace(c, WS_FXO, 2 * n * fb);
  void* Ye = dwf_workspace(c, WS_FYE, 2 * n * fb);
  void* Yo = dwf_workspace(c, WS_FYO, 2 * n * fb);
  if (!Xe || !Xo || !Ye || !Yo) return dwf_fail(c, DWF_ENOMEM, "force workspace");
  std::vector<double> mass(2 * n);
  ForceCoef coef;
  for (int f = 0; f < DWF_MAX_RHS; f++) coef.c[f] = 0.0;
  for (int i = 0; i < n; i++) {
    mass[i] = m1[i];
    mass[n + i] = m2[i];
    coef.c[i] = 1.0;
    coef.c[n + i] = -1.0;
  }
  // pairs 0..n-1: (X, M1 X) at m1; pairs n..2n-1: (X, phi) at m2
  DWF_CUDA(c, cudaMemcpyAsync(Xe, X, n * fb, cudaMemcpyDeviceToDevice, st));
  DWF_CUDA(c, cudaMemcpyAsync((char*)Xe + n * fb, X, n * fb, cudaMemcpyDeviceToDevice, st));
  DWF_CUDA(c, cudaMemcpyAsync((char*)Ye + n * fb, phi, n * fb, cudaMemcpyDeviceToDevice, st));
  rc = mpc_apply(c, Ye, X, Xo, mass.data(), 0, prec, n, 0, st, nullptr);  // M1 X, and M_oo^-1 M_oe X at m1
  if (rc) return rc;
  {  // M_oo^-1 M_oe X at m2
    HopLaunch hx;
    memset(&hx, 0, sizeof(hx));
    hx.out = (char*)Xo + n * fb;
    hx.in = X;
    hx.out_parity = 1;
    hx.nrhs = n;
    hx.alpha = -0.5;
    hx.inv_mode = 1;
    hx.mf = mass.data() + n;
    rc = launch_hop(c, hx, prec, st, nullptr);
    if (rc) return rc;
  }
  return force_tail(c, force, Xe, Xo, true, Ye, Yo, mass.data(), coef, 2 * n, prec, st);
}

// S = sum_i [2 Re <phi_i, X_i> - |M_pc(mf_i) X_i|^2] (the variational
// estimator of phi^dag (M^dag M)^-1 phi, error quadratic in the solve's).
extern "C" int dwf_pf_action(dwf_ctx* c, double* S, const void* phi, const void* X, const double* mf, int npf,
                             void* stream) {
  if (!c || !S || !phi || !X || !mf || npf < 1) return DWF_EINVAL;
  if (npf > DWF_MAX_RHS) return dwf_fail(c, DWF_EINVAL, "npf out of range");
  if (!dwf_is_device_ptr(phi) || !dwf_is_device_ptr(X)) return dwf_fail(c, DWF_EINVAL, "device buffers required");
  if (((uintptr_t)phi & 15) || ((uintptr_t)X & 15)) return dwf_fail(c, DWF_EINVAL, "alignment");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t he = c->g.Vh * 12 * c->g.Ls;
  const size_t bytes = (size_t)npf * he * 16;
  void* Xo = dwf_workspace(c, WS_FXO, bytes);
  void* Y = dwf_workspace(c, WS_FYE, bytes);
  if (!Xo || !Y) return dwf_fail(c, DWF_ENOMEM, "workspace");
  int np = 0;
  int rc = blas_cdot_partials(c, phi, X, npf * he, DWF_F64, st, &np);
  if (rc) return rc;
  rc = blas_finalize(c, np, 2, S_TMP0, st);
  if (rc) return rc;
  rc = mpc_apply(c, Y, X, Xo, mf, 0, DWF_F64, npf, 1, st, &np);  // |M X|^2 partials of every field
  if (rc) return rc;
  rc = blas_finalize(c, np, 1, S_TMP2, st);
  if (rc) return rc;
  rc = read_scalars(c, S_TMP0, 3, st);
  if (rc) return rc;
  *S = 2.0 * c->hscal[S_TMP0] - c->hscal[S_TMP2];
  if (!isfinite(*S)) return dwf_fail(c, DWF_ENAN, "action is not finite");
  DWF_CUDA(c, cudaGetLastError());
  return DWF_OK;
}
