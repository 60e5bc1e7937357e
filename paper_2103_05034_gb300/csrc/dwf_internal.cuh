// Internal declarations of the GB300 DWF multigrid library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/dwfmg.h"

#define DWF_MAX_RHS 64
// Internal precision tag of the hopping kernel with FP64 storage and
// float-float arithmetic (dfloat.cuh); not an ABI precision.
#define DWF_P_DF 7
#define DWF_NWS 40  // workspace slots
#define CG_SMALL_BYTES 384  // status and barrier counters of the persistent coarse CG

// ------------------------------------------------------------------ complex helpers
template <class R>
struct cpx {
  R re, im;
};

template <class R>
__device__ __forceinline__ cpx<R> cmake(R a, R b) {
  cpx<R> z;
  z.re = a;
  z.im = b;
  return z;
}

// Storage traits: element type of a complex number in memory and the real
// type used for arithmetic.
template <int P>
struct Prec;
template <>
struct Prec<DWF_F64> {
  typedef double2 S;  // stored complex
  typedef double R;   // arithmetic
  typedef double2 LS; // stored link element
};
template <>
struct Prec<DWF_F32> {
  typedef float2 S;
  typedef float R;
  typedef float2 LS;
};
template <>
struct Prec<DWF_F16S> {
  typedef __half2 S;
  typedef float R;
  typedef float2 LS;
};

__device__ __forceinline__ cpx<double> ld_c(const double2* p) {
  double2 v = *p;
  return cmake(v.x, v.y);
}
__device__ __forceinline__ cpx<float> ld_c(const float2* p) {
  float2 v = *p;
  return cmake(v.x, v.y);
}
__device__ __forceinline__ cpx<float> ld_c(const __half2* p) {
  float2 v = __half22float2(*p);
  return cmake(v.x, v.y);
}
__device__ __forceinline__ void st_c(double2* p, cpx<double> z) { *p = make_double2(z.re, z.im); }
__device__ __forceinline__ void st_c(float2* p, cpx<float> z) { *p = make_float2(z.re, z.im); }
__device__ __forceinline__ void st_c(__half2* p, cpx<float> z) {
  *p = __floats2half2_rn(z.re, z.im);
}

// Per-thread partial sum for reductions.  FP64 data accumulate in FP64; FP32
// and FP16-storage data accumulate in FP32 with a compensation term (Kahan's
// summation: the rounding error of every addition is carried to the next),
// and the partials of all threads are combined in FP64.  GB300 runs FP64 at a
// small fraction of its FP32 rate, so a per-element FP64 sum would cost more
// ALU time than the memory traffic of the pass.
template <class R>
struct PartialSum;
template <>
struct PartialSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct PartialSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ------------------------------------------------------------------ geometry
struct Geom {
  int L[4];   // Lx, Ly, Lz, Lt
  int Lxh;    // Lx / 2
  int64_t Vh; // sites per parity
  int Ls;
};

// Fifth-dimension coefficients of M (Eq. 4) for one mass: d = 5 - M5,
// kappa = 1/(1 + m d^-Ls), dls1 = d^(1-Ls).
struct FifthCoef {
  double m, kappa, dls1;
};

// ------------------------------------------------------------------ context
struct dwf_ctx {
  Geom g;
  double M5;
  int device;
  // parity-split, double-stored links: links[p] is [Vh][8][3][3] complex,
  // slot 2mu = U_mu(x), slot 2mu+1 = U_mu(x-mu)^dag, for sites x of parity p.
  double2* links64[2];
  float2* links32[2];
  // workspace (grown on demand)
  void* ws[DWF_NWS];
  size_t ws_bytes[DWF_NWS];
  double* partials;   // reduction partials
  size_t partials_n;
  double* dscal;      // device scalars for solvers
  double* hscal;      // pinned host mirror
  int hop_variant[3]; // tuned hopping-kernel variant per precision
  int f64_arith;      // FP64 hopping launches: DWF_ARITH_FP64 or DWF_ARITH_FLOAT_FLOAT
  double hop_l2_budget[3];  // L2 bytes the z-chunked traversal plans for (0: 48 MB)
  int64_t launches;   // kernel launches since the last counter reset
  double hop_bytes;   // algorithmic bytes of hopping-term launches
  std::string err;
};

// Error helpers (host).
int dwf_fail(dwf_ctx* c, int code, const std::string& msg);
int dwf_cuda_check(dwf_ctx* c, cudaError_t e, const char* where);
#define DWF_CUDA(ctx, call)                                         \
  do {                                                              \
    cudaError_t _e = (call);                                        \
    if (_e != cudaSuccess) return dwf_cuda_check((ctx), _e, #call); \
  } while (0)

size_t dwf_complex_bytes(int prec);
// A context on the same lattice and links with fifth-dimension extent ls (api.cu).
int dwf_ctx_clone_ls(const dwf_ctx* src, int ls, dwf_ctx** out, cudaStream_t st);
void* dwf_workspace(dwf_ctx* c, int slot, size_t bytes);
void dwf_ws_release(dwf_ctx* c, int slot);  // free one workspace slot (mg.cu)
bool dwf_is_device_ptr(const void* p);

// ------------------------------------------------------------------ launchers
// Hopping-term launch descriptor with the fused fifth-dimension epilogue:
//   v   = alpha * D_hop^{(dagger)} in                      (hop part)
//   v  += aux term: aux, M aux or M^dag aux                (aux_mode 1,2,3)
//   v   = M^-1 v or M^-dag v                               (inv_mode 1,2)
//   out = v, or Gamma_5 v (gamma_5 and s -> Ls-1-s)        (g5r5)
//   partials[block] += |v|^2                               (reduce)
struct HopLaunch {
  void* out;
  const void* in;
  const void* aux;
  int out_parity;
  int dagger;
  int nrhs;
  int64_t rhs_stride;  // complex elements between consecutive rhs fields
  double alpha;
  int aux_mode;        // 0 none, 1 aux, 2 M aux, 3 M^dag aux
  int inv_mode;        // 0 none, 1 M^-1, 2 M^-dag
  int g5r5;
  int reduce;          // 1: |out|^2 partials into ctx->partials
  const double* mf;    // host array [nrhs] of masses (aux_mode>=2 or inv_mode>0)
  // fused CG update instead of storing out: x += alpha p, r -= alpha out,
  // |r|^2 reduced (alpha = device scalar); requires reduce = 1
  void* cg_x;
  void* cg_r;
  const void* cg_p;
  const double* cg_alpha;
  int cg_alpha_stride;  // doubles between consecutive rhs' alpha (0: shared)
  int cg_x32;          // x is FP32 whatever the field precision (FP16-storage CG)
  // fused Chebyshev recurrence step instead of storing out (cheb_tp set):
  // tp = ta out + tb x - tp, acc += cacc tp (acc may be null); same layout as out
  const void* cheb_x;
  void* cheb_tp;
  void* cheb_acc;
  double cheb_ta, cheb_tb, cheb_cacc;
};

// The Chebyshev step fused into the last hopping launch of an operator
// application (ddw_apply): tp = ta (A x) + tb x - tp; acc += cacc tp.
struct ChebFuse {
  const void* x;
  void* tp;
  void* acc;
  double ta, tb, cacc;
};

int launch_hop(dwf_ctx* c, const HopLaunch& h, int prec, cudaStream_t st, int* nblocks);
int launch_mooee(dwf_ctx* c, void* out, const void* in, const double* mf, int dagger, int inverse,
                 int prec, int nrhs, int64_t rhs_stride, cudaStream_t st);

// BLAS-1 (blas.cu).  n = number of complex elements.
int blas_norm2_partials(dwf_ctx* c, const void* a, int64_t n, int prec, cudaStream_t st, int* nparts);
int blas_cdot_partials(dwf_ctx* c, const void* a, const void* b, int64_t n, int prec,
                       cudaStream_t st, int* nparts);
// Sum nparts partials (width 1 or 2 doubles) into dscal[dst..dst+width-1].
int blas_finalize(dwf_ctx* c, int nparts, int width, int dst, cudaStream_t st);
// As blas_finalize, then mode 1: alpha = rr/pAp; mode 2: beta = rrnew/rr, rr = rrnew.
int blas_finalize_mode(dwf_ctx* c, int nparts, int width, int dst, int mode, cudaStream_t st, int base = 0);
// Grow the reduction-partials buffer to at least n doubles.
int dwf_reserve_partials(dwf_ctx* c, size_t n);
// y = a*x + b*y with real host scalars, any precisions (x, y may differ).
int blas_axpby(dwf_ctx* c, double a, const void* x, int px, double b, void* y, int py, int64_t n,
               cudaStream_t st);
// y = x converted between precisions.
int blas_copy(dwf_ctx* c, void* y, int py, const void* x, int px, int64_t n, cudaStream_t st);
// CG updates with device scalars (dscal indices), precision prec:
//   x += alpha p; r -= alpha Ap; partials |r|^2
int blas_cg_xr(dwf_ctx* c, void* x, void* r, const void* p, const void* Ap, int64_t n, int prec,
               int ialpha, cudaStream_t st, int* nparts);
//   p = r + beta p
int blas_cg_p(dwf_ctx* c, void* p, const void* r, int64_t n, int prec, int ibeta, cudaStream_t st);
// Batched forms over nseg consecutive vectors of n elements each, segment i
// using the scalar bank dscal[S_BANK0 + i * S_BANK]:
//   p_i = r_i + beta_i p_i
int blas_cg_p_batch(dwf_ctx* c, void* p, const void* r, int64_t n, int nseg, int prec, cudaStream_t st);
//   sum the partials of each segment (nparts_per consecutive doubles) into its
//   bank slot dst, then mode 1: alpha = rr/pAp; 2: beta = rrnew/rr, rr = rrnew;
//   mode 0: the sums only
int blas_finalize_batch(dwf_ctx* c, int nparts_per, int nseg, int dst, int mode, cudaStream_t st);
// Exchange the contents of two device buffers (16-byte aligned, bytes % 16 == 0).
int blas_swap(dwf_ctx* c, void* a, void* b, size_t bytes, cudaStream_t st);
// z = a x + b y + c z (same precision)
int blas_axpbypcz(dwf_ctx* c, double a, const void* x, double b, const void* y, double cz, void* z,
                  int64_t n, int prec, cudaStream_t st);
// Chebyshev recurrence step: tp = ta*Ax + tb*x - tp; acc += cacc*tp (acc may be NULL)
int blas_cheb_step(dwf_ctx* c, void* tp, const void* Ax, const void* x, double ta, double tb, void* acc,
                   double cacc, int64_t n, int prec, cudaStream_t st);
// y += (ar + i ai) x, precisions (F64|F32) x (F64|F32)
int blas_caxpy(dwf_ctx* c, double ar, double ai, const void* x, int px, void* y, int py, int64_t n,
               cudaStream_t st);
// Full-lattice D_DW / D_DW^dag / H_DW (g5 = 1) on nrhs full fields (api.cu);
// with cf the result is not stored but folded into cf's Chebyshev step.
int ddw_apply(dwf_ctx* c, void* out, const void* in, const double* mf, int dagger, int g5, int prec,
              int nrhs, cudaStream_t st, const ChebFuse* cf = nullptr);
int norm2_dev(dwf_ctx* c, const void* a, int64_t n, int prec, int dst, cudaStream_t st);
// M_pc (dagger 0) or M_pc^dag (1) of nrhs even fields; tmp receives the odd
// intermediate M_oo^-1 M_oe in (or its dagger form); reduce = |out|^2 partials.
int mpc_apply(dwf_ctx* c, void* out, const void* in, void* tmp, const double* mf, int dagger, int prec,
              int nrhs, int reduce, cudaStream_t st, int* nparts);
int read_scalars(dwf_ctx* c, int first, int n, cudaStream_t st);
// dscal[dst] = dscal[num] / dscal[den]
int blas_scalar_div(dwf_ctx* c, int dst, int num, int den, cudaStream_t st);


// Workspace slots of the red-black solvers (single and batched) and the
// force.  The MG setup uses 16..27, the autotuner 30..31.
enum {
  WS_B = 2,      // full FP64 source (host input)
  WS_X = 3,      // full FP64 solution (host output)
  WS_BP = 4,     // even FP64 b'_e
  WS_RHS = 5,    // even FP64 M_pc^dag b'_e
  WS_RHI = 6,    // even FP64 residual / scratch
  WS_YHI = 7,    // even FP64 temporary
  WS_OHI = 8,    // odd FP64 temporary
  WS_XLO = 9,    // even inner x
  WS_RLO = 10,   // even inner r
  WS_P = 11,     // even p
  WS_AP = 12,    // even Ap
  WS_YLO = 13,   // even y = M_pc p
  WS_OLO = 14,   // odd temporary
  WS_FULL = 15,  // full FP64 temporary (true residual)
  WS_BE = 32,    // batched solve: sources split by parity, [nrhs][half]
  WS_BO = 33,
  WS_XE = 34,    // batched solve: solutions split by parity
  WS_XO = 35,
  WS_FXO = 36,   // force: X_o, Y_e, Y_o of all pseudofermions
  WS_FYE = 37,
  WS_FYO = 38,
  WS_FXE = 39    // ratio force: X twice (one copy per bilinear)
};

// Device scalar slots.
enum {
  S_RR = 0,    // |r|^2
  S_PAP = 1,   // <p, A p>
  S_ALPHA = 2,
  S_BETA = 3,
  S_RRNEW = 4,
  S_TMP0 = 8,
  S_TMP1 = 9,
  S_TMP2 = 10,
  S_TMP3 = 11,
  // batched CG: slot i owns the bank dscal[S_BANK0 + i * S_BANK .. +S_BANK-1]
  // with the offsets S_RR .. S_RRNEW above plus these (bank-relative)
  S_BT0 = 6,
  S_BT1 = 7,
  S_BDOT = 8,  // two doubles: <r, p>
  S_BANK0 = 32,
  S_BANK = 10,
  S_NSCAL = S_BANK0 + S_BANK * DWF_MAX_RHS
};
