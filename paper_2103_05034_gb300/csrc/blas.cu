// BLAS-1 kernels with FP64 accumulation for global sums (the inner products
// of every Krylov step, arXiv:2103.05034 Secs. 3 and 5.1); single-precision
// data accumulate per thread in compensated FP32 (PartialSum) and combine in
// FP64.  Reductions are
// two-pass and deterministic: a fixed grid writes one partial per CTA (warp
// shuffles, then shared memory), one CTA sums the partials in order.
#include "dwf_internal.cuh"

namespace {

constexpr int BT = 256;          // threads per CTA
constexpr int BLAS_BLOCKS = 1216; // 8 CTAs per SM on 152 SMs

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += sh[i];
  }
  __syncthreads();
  return t;
}

template <int P>
__global__ void __launch_bounds__(BT) k_norm2(const typename Prec<P>::S* a, long long n, double* part) {
  typedef typename Prec<P>::R R;
  __shared__ double sh[BT / 32];
  PartialSum<R> acc;
  for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
    const auto z = ld_c(a + i);
    acc.add(fma(z.re, z.re, z.im * z.im));
  }
  const double t = block_sum(acc.value(), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

template <int P>
__global__ void __launch_bounds__(BT) k_cdot(const typename Prec<P>::S* a, const typename Prec<P>::S* b,
                                             long long n, double* part) {
  typedef typename Prec<P>::R R;
  __shared__ double sh[BT / 32];
  PartialSum<R> pre, pim;
  for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
    const auto x = ld_c(a + i);
    const auto y = ld_c(b + i);
    pre.add(fma(x.re, y.re, x.im * y.im));
    pim.add(fma(x.re, y.im, -(x.im * y.re)));
  }
  const double re = pre.value(), im = pim.value();
  const double tr = block_sum(re, sh);
  const double ti = block_sum(im, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = tr;
    part[2 * blockIdx.x + 1] = ti;
  }
}

// mode 0: dscal[dst..] = sums; 1: alpha = rr/pAp after storing pAp;
// 2: beta = rrnew/rr, rr = rrnew after storing rrnew.
__global__ void __launch_bounds__(BT) k_finalize(const double* part, int n, int width, double* dscal,
                                                 int dst, int mode, int base) {
  __shared__ double sh[BT / 32];
  for (int k = 0; k < width; k++) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += BT) acc += part[(size_t)i * width + k];
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) dscal[dst + k] = t;
  }
  if (threadIdx.x == 0) {
    double* q = dscal + base;
    if (mode == 1) {
      q[S_ALPHA] = q[S_RR] / q[S_PAP];
    } else if (mode == 2) {
      q[S_BETA] = q[S_RRNEW] / q[S_RR];
      q[S_RR] = q[S_RRNEW];
    }
  }
}

// Batched finalize: CTA i sums the n partials part[i * n ..] into bank i.
__global__ void __launch_bounds__(BT) k_finalize_batch(const double* part, int n, double* dscal, int dst,
                                                       int mode) {
  __shared__ double sh[BT / 32];
  const double* pi = part + (size_t)blockIdx.x * n;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += BT) acc += pi[i];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    double* q = dscal + S_BANK0 + blockIdx.x * S_BANK;
    q[dst] = t;
    if (mode == 1) {
      q[S_ALPHA] = q[S_RR] / q[S_PAP];
    } else if (mode == 2) {
      q[S_BETA] = q[S_RRNEW] / q[S_RR];
      q[S_RR] = q[S_RRNEW];
    }
  }
}

// Exchange two buffers of n 16-byte words.
__global__ void __launch_bounds__(BT) k_swap(uint4* a, uint4* b, long long n) {
  for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
    const uint4 t = a[i];
    a[i] = b[i];
    b[i] = t;
  }
}

template <int PX, int PY>
__global__ void __launch_bounds__(BT) k_axpby(double a, const typename Prec<PX>::S* x, double b,
                                              typename Prec<PY>::S* y, long long n) {
  typedef typename Prec<PY>::R RY;
  for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
    const auto xv = ld_c(x + i);
    cpx<RY> o;
    if (PX != DWF_F64 && PY != DWF_F64) {  // single-precision data: FP32 arithmetic
      const float af = (float)a, bf = (float)b;
      if (b == 0.0) {
        o.re = af * (float)xv.re;
        o.im = af * (float)xv.im;
      } else {
        const auto yv = ld_c(y + i);
        o.re = fmaf(af, (float)xv.re, bf * (float)yv.re);
        o.im = fmaf(af, (float)xv.im, bf * (float)yv.im);
      }
    } else if (b == 0.0) {
      o.re = (RY)(a * (double)xv.re);
      o.im = (RY)(a * (double)xv.im);
    } else {
      const auto yv = ld_c(y + i);
      o.re = (RY)(a * (double)xv.re + b * (double)yv.re);
      o.im = (RY)(a * (double)xv.im + b * (double)yv.im);
    }
    st_c(y + i, o);
  }
}

template <int P>
__global__ void __launch_bounds__(BT) k_cg_xr(typename Prec<P>::S* x, typename Prec<P>::S* r,
                                              const typename Prec<P>::S* p,
                                              const typename Prec<P>::S* Ap, long long n,
                                              const double* dscal, int ialpha, double* part) {
  typedef typename Prec<P>::R R;
  __shared__ double sh[BT / 32];
  const R alpha = (R)dscal[ialpha];
  PartialSum<R> acc;
  for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
    auto xv = ld_c(x + i);
    auto rv = ld_c(r + i);
    const auto pv = ld_c(p + i);
    const auto av = ld_c(Ap + i);
    xv.re = fma(alpha, pv.re, xv.re);
    xv.im = fma(alpha, pv.im, xv.im);
    rv.re = fma(-alpha, av.re, rv.re);
    rv.im = fma(-alpha, av.im, rv.im);
    st_c(x + i, xv);
    st_c(r + i, rv);
    acc.add(fma(rv.re, rv.re, rv.im * rv.im));
  }
  const double t = block_sum(acc.value(), sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// p = r + beta p; segment blockIdx.y (n elements) takes dscal[ibeta + y * bstride]
template <int P>
__global__ void __launch_bounds__(BT) k_cg_p(typename Prec<P>::S* p, const typename Prec<P>::S* r,
                                             long long n, const double* dscal, int ibeta, int bstride) {
  typedef typename Prec<P>::R R;
  const R beta = (R)dscal[ibeta + blockIdx.y * bstride];
  p += (size_t)blockIdx.y * n;
  r += (size_t)blockIdx.y * n;
  for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
    auto pv = ld_c(p + i);
    const auto rv = ld_c(r + i);
    pv.re = fma(beta, pv.re, rv.re);
    pv.im = fma(beta, pv.im, rv.im);
    st_c(p + i, pv);
  }
}

template <int P>
__global__ void __launch_bounds__(BT) k_axpbypcz(double a, const typename Prec<P>::S* x, double b,
                                                 const typename Prec<P>::S* y, double cz,
                                                 typename Prec<P>::S* z, long long n) {
  typedef typename Prec<P>::R R;
  for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
    const auto xv = ld_c(x + i);
    const auto yv = ld_c(y + i);
    cpx<R> o;
    o.re = (R)a * xv.re + (R)b * yv.re;
    o.im = (R)a * xv.im + (R)b * yv.im;
    if (cz != 0.0) {  // z is not read when its coefficient is zero (it may be uninitialised)
      const auto zv = ld_c(z + i);
      o.re += (R)cz * zv.re;
      o.im += (R)cz * zv.im;
    }
    st_c(z + i, o);
  }
}

// Chebyshev step: tp <- ta * Ax + tb * x - tp (the next T), acc += cacc * tp.
template <int P>
__global__ void __launch_bounds__(BT) k_cheb_step(typename Prec<P>::S* tp, const typename Prec<P>::S* Ax,
                                                  const typename Prec<P>::S* x, double ta, double tb,
                                                  typename Prec<P>::S* acc, double cacc, long long n) {
  typedef typename Prec<P>::R R;
  for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
    const auto av = ld_c(Ax + i);
    const auto xv = ld_c(x + i);
    const auto pv = ld_c(tp + i);
    cpx<R> o;
    o.re = (R)ta * av.re + (R)tb * xv.re - pv.re;
    o.im = (R)ta * av.im + (R)tb * xv.im - pv.im;
    st_c(tp + i, o);
    if (acc) {
      auto cv = ld_c(acc + i);
      cv.re += (R)cacc * o.re;
      cv.im += (R)cacc * o.im;
      st_c(acc + i, cv);
    }
  }
}

// y += (ar + i ai) x, any precision pair.
template <int PX, int PY>
__global__ void __launch_bounds__(BT) k_caxpy(double ar, double ai, const typename Prec<PX>::S* x,
                                              typename Prec<PY>::S* y, long long n) {
  typedef typename Prec<PY>::R RY;
  for (long long i = (long long)blockIdx.x * BT + threadIdx.x; i < n; i += (long long)gridDim.x * BT) {
    const auto xv = ld_c(x + i);
    const auto yv = ld_c(y + i);
    cpx<RY> o;
    if (PX != DWF_F64 && PY != DWF_F64) {  // single-precision data: FP32 arithmetic
      const float arf = (float)ar, aif = (float)ai;
      o.re = fmaf(arf, (float)xv.re, fmaf(-aif, (float)xv.im, (float)yv.re));
      o.im = fmaf(arf, (float)xv.im, fmaf(aif, (float)xv.re, (float)yv.im));
    } else {
      o.re = (RY)((double)yv.re + ar * xv.re - ai * xv.im);
      o.im = (RY)((double)yv.im + ar * xv.im + ai * xv.re);
    }
    st_c(y + i, o);
  }
}

__global__ void k_div(double* dscal, int dst, int num, int den) { dscal[dst] = dscal[num] / dscal[den]; }

int grid_for(long long n) {
  long long g = (n + BT - 1) / BT;
  if (g > BLAS_BLOCKS) g = BLAS_BLOCKS;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

#define DWF_PREC_SWITCH(prec, CALL)                   \
  switch (prec) {                                     \
    case DWF_F64: {                                   \
      constexpr int P = DWF_F64;                      \
      CALL;                                           \
    } break;                                          \
    case DWF_F32: {                                   \
      constexpr int P = DWF_F32;                      \
      CALL;                                           \
    } break;                                          \
    case DWF_F16S: {                                  \
      constexpr int P = DWF_F16S;                     \
      CALL;                                           \
    } break;                                          \
    default:                                          \
      return dwf_fail(c, DWF_EINVAL, "bad precision"); \
  }

int blas_norm2_partials(dwf_ctx* c, const void* a, int64_t n, int prec, cudaStream_t st, int* nparts) {
  const int g = grid_for(n);
  c->launches++;
  DWF_PREC_SWITCH(prec, (k_norm2<P><<<g, BT, 0, st>>>((const typename Prec<P>::S*)a, n, c->partials)));
  *nparts = g;
  return DWF_OK;
}

int blas_cdot_partials(dwf_ctx* c, const void* a, const void* b, int64_t n, int prec, cudaStream_t st,
                       int* nparts) {
  const int g = grid_for(n);
  c->launches++;
  DWF_PREC_SWITCH(prec, (k_cdot<P><<<g, BT, 0, st>>>((const typename Prec<P>::S*)a,
                                                       (const typename Prec<P>::S*)b, n, c->partials)));
  *nparts = g;
  return DWF_OK;
}

int blas_finalize_mode(dwf_ctx* c, int nparts, int width, int dst, int mode, cudaStream_t st, int base) {
  c->launches++;
  k_finalize<<<1, BT, 0, st>>>(c->partials, nparts, width, c->dscal, dst, mode, base);
  return DWF_OK;
}

int blas_finalize(dwf_ctx* c, int nparts, int width, int dst, cudaStream_t st) {
  return blas_finalize_mode(c, nparts, width, dst, 0, st);
}

int blas_axpby(dwf_ctx* c, double a, const void* x, int px, double b, void* y, int py, int64_t n,
               cudaStream_t st) {
  const int g = grid_for(n);
  c->launches++;
#define DWF_AXPBY(PXV, PYV)                                                                        \
  if (px == PXV && py == PYV) {                                                                   \
    k_axpby<PXV, PYV><<<g, BT, 0, st>>>(a, (const typename Prec<PXV>::S*)x, b,                     \
                                         (typename Prec<PYV>::S*)y, n);                            \
    return DWF_OK;                                                                                \
  }
  DWF_AXPBY(DWF_F64, DWF_F64)
  DWF_AXPBY(DWF_F64, DWF_F32)
  DWF_AXPBY(DWF_F64, DWF_F16S)
  DWF_AXPBY(DWF_F32, DWF_F64)
  DWF_AXPBY(DWF_F32, DWF_F32)
  DWF_AXPBY(DWF_F32, DWF_F16S)
  DWF_AXPBY(DWF_F16S, DWF_F64)
  DWF_AXPBY(DWF_F16S, DWF_F32)
  DWF_AXPBY(DWF_F16S, DWF_F16S)
#undef DWF_AXPBY
  return dwf_fail(c, DWF_EINVAL, "bad precision pair");
}

int blas_copy(dwf_ctx* c, void* y, int py, const void* x, int px, int64_t n, cudaStream_t st) {
  return blas_axpby(c, 1.0, x, px, 0.0, y, py, n, st);
}

int blas_cg_xr(dwf_ctx* c, void* x, void* r, const void* p, const void* Ap, int64_t n, int prec,
               int ialpha, cudaStream_t st, int* nparts) {
  const int g = grid_for(n);
  c->launches++;
  DWF_PREC_SWITCH(prec, (k_cg_xr<P><<<g, BT, 0, st>>>(
                            (typename Prec<P>::S*)x, (typename Prec<P>::S*)r,
                            (const typename Prec<P>::S*)p, (const typename Prec<P>::S*)Ap, n,
                            c->dscal, ialpha, c->partials)));
  *nparts = g;
  return DWF_OK;
}

int blas_cg_p(dwf_ctx* c, void* p, const void* r, int64_t n, int prec, int ibeta, cudaStream_t st) {
  const int g = grid_for(n);
  c->launches++;
  DWF_PREC_SWITCH(prec, (k_cg_p<P><<<g, BT, 0, st>>>((typename Prec<P>::S*)p,
                                                       (const typename Prec<P>::S*)r, n, c->dscal,
                                                       ibeta, 0)));
  return DWF_OK;
}

int blas_cg_p_batch(dwf_ctx* c, void* p, const void* r, int64_t n, int nseg, int prec, cudaStream_t st) {
  if (nseg < 1 || nseg > DWF_MAX_RHS) return dwf_fail(c, DWF_EINVAL, "nseg out of range");
  int g = grid_for(n) / nseg;
  if (g < 64) g = 64;
  c->launches++;
  DWF_PREC_SWITCH(prec, (k_cg_p<P><<<dim3(g, nseg), BT, 0, st>>>((typename Prec<P>::S*)p,
                                                                   (const typename Prec<P>::S*)r, n,
                                                                   c->dscal, S_BANK0 + S_BETA, S_BANK)));
  return DWF_OK;
}

int blas_finalize_batch(dwf_ctx* c, int nparts_per, int nseg, int dst, int mode, cudaStream_t st) {
  if (nseg < 1 || nseg > DWF_MAX_RHS) return dwf_fail(c, DWF_EINVAL, "nseg out of range");
  c->launches++;
  k_finalize_batch<<<nseg, BT, 0, st>>>(c->partials, nparts_per, c->dscal, dst, mode);
  return DWF_OK;
}

int blas_swap(dwf_ctx* c, void* a, void* b, size_t bytes, cudaStream_t st) {
  if ((bytes & 15) || ((uintptr_t)a & 15) || ((uintptr_t)b & 15))
    return dwf_fail(c, DWF_EINVAL, "swap needs 16-byte aligned buffers and sizes");
  if (a == b || bytes == 0) return DWF_OK;
  const long long n = (long long)(bytes / 16);
  c->launches++;
  k_swap<<<grid_for(n), BT, 0, st>>>((uint4*)a, (uint4*)b, n);
  return DWF_OK;
}

int blas_axpbypcz(dwf_ctx* c, double a, const void* x, double b, const void* y, double cz, void* z,
                  int64_t n, int prec, cudaStream_t st) {
  const int g = grid_for(n);
  c->launches++;
  DWF_PREC_SWITCH(prec, (k_axpbypcz<P><<<g, BT, 0, st>>>(a, (const typename Prec<P>::S*)x, b,
                                                           (const typename Prec<P>::S*)y, cz,
                                                           (typename Prec<P>::S*)z, n)));
  return DWF_OK;
}

int blas_cheb_step(dwf_ctx* c, void* tp, const void* Ax, const void* x, double ta, double tb, void* acc,
                   double cacc, int64_t n, int prec, cudaStream_t st) {
  const int g = grid_for(n);
  c->launches++;
  DWF_PREC_SWITCH(prec, (k_cheb_step<P><<<g, BT, 0, st>>>((typename Prec<P>::S*)tp,
                                                            (const typename Prec<P>::S*)Ax,
                                                            (const typename Prec<P>::S*)x, ta, tb,
                                                            (typename Prec<P>::S*)acc, cacc, n)));
  return DWF_OK;
}

int blas_caxpy(dwf_ctx* c, double ar, double ai, const void* x, int px, void* y, int py, int64_t n,
               cudaStream_t st) {
  const int g = grid_for(n);
  c->launches++;
#define DWF_CAXPY(PXV, PYV)                                                                         \
  if (px == PXV && py == PYV) {                                                                    \
    k_caxpy<PXV, PYV><<<g, BT, 0, st>>>(ar, ai, (const typename Prec<PXV>::S*)x,                    \
                                         (typename Prec<PYV>::S*)y, n);                             \
    return DWF_OK;                                                                                 \
  }
  DWF_CAXPY(DWF_F64, DWF_F64)
  DWF_CAXPY(DWF_F32, DWF_F64)
  DWF_CAXPY(DWF_F32, DWF_F32)
  DWF_CAXPY(DWF_F64, DWF_F32)
#undef DWF_CAXPY
  return dwf_fail(c, DWF_EINVAL, "bad precision pair");
}

int blas_scalar_div(dwf_ctx* c, int dst, int num, int den, cudaStream_t st) {
  c->launches++;
  k_div<<<1, 1, 0, st>>>(c->dscal, dst, num, den);
  return DWF_OK;
}
