// Persistent coarse-grid CG (Sec. 3.4: the coarse system of the HDCR V-cycle
// is solved by CG on the normal equations of the hermitian little Dirac
// operator A, here A^2 e = A r, to a loose relative tolerance).
//
// The coarse grid is small (a few thousand sites x nb), so a kernel-per-step
// CG is bound by launch and host-synchronisation latency, not by the A
// traffic.  This file runs the whole solve as ONE cooperative launch: every
// CTA owns a slice of the coarse rows, the grid meets at a software barrier
// twice per iteration, and the scalars are formed redundantly by every CTA
// from per-CTA partial sums (fixed summation order, so all CTAs take the same
// convergence decision and the result is deterministic).
//
// Matrix-vector product: one warp per output row (site x, row j); lane k
// reads A_d(x)[j][k] (nb consecutive complex numbers, coalesced) and the
// neighbour vector element v(x+d)[k]; a warp reduction forms the row.
//
// Iteration (p is double-buffered so that it can be formed on the fly):
//   phase A: p_i = r + beta p_{i-1} (gathered at the neighbours), t = A p_i,
//            owners store p_i;  partial |t|^2               -> barrier
//   phase B: alpha = rr / |t|^2;  q = A t;  e += alpha p_i,
//            r -= alpha q (own rows);  partial |r|^2        -> barrier
//   beta = |r_new|^2 / rr; stop when |r_new|^2 <= tol^2 |A r_0|^2.
// Every wait is bounded: a CTA that gives up sets an error flag and returns,
// so the others give up too and the host reads DWF_ETIMEOUT.
#include "dwf_internal.cuh"
#include "mg_kernels.cuh"

namespace {

constexpr int CG_THREADS = 256;
constexpr int CG_WARPS = CG_THREADS / 32;
constexpr unsigned CG_SPIN = 1u << 22;  // polls per barrier before giving up

enum { ST_ITERS = 0, ST_ERR = 1 };
enum { ERR_TIMEOUT = 1, ERR_NAN = 2 };

struct CoarseCGArgs {
  const float2* A;  // [nc][9][nb][nb]
  int Lc[4];
  int nc, nb;
  const float2* rhs;
  float2 *e, *r, *p0, *p1, *t;
  double* part;        // [nblk] partial sums of the current reduction
  double* tot;         // [2] grid totals (alternating)
  unsigned* bar;       // arrival counter, zero at launch
  unsigned* rel;       // release counter, zero at launch
  int* status;         // [ST_ITERS], [ST_ERR]
  int* acc;            // optional: [0] += iterations, [1] |= error (sticky over launches)
  double tol2;
  int maxiter;
};

__device__ void set_err(const CoarseCGArgs& a, int code) {
  atomicCAS(&a.status[ST_ERR], 0, code);
  if (a.acc) atomicOr(&a.acc[1], code);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Grid-wide sum at barrier number k (k = 1, 2, ...).  Every CTA adds its
// partial (lane 0 of each warp holds the warp's) to part[blockIdx]; the CTA
// that arrives last sums all partials in block order (fixed order, so the
// result does not depend on which CTA is last) into tot[k & 1] and releases
// the others, which wait on rel >= k.  Returns false when a wait ran out or
// another CTA has given up (the error is recorded).
__device__ bool reduce_barrier(const CoarseCGArgs& a, unsigned k, double warp_partial, double* total) {
  __shared__ double w[CG_WARPS];
  __shared__ int flag;
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = warp_partial;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < CG_WARPS; i++) s += w[i];
    a.part[blockIdx.x] = s;
    __threadfence();
    const unsigned old = atomicAdd(a.bar, 1u);
    flag = (old == k * gridDim.x - 1) ? 2 : 0;  // 2: this CTA is the last to arrive
  }
  __syncthreads();
  if (flag == 2) {
    __threadfence();
    double v = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += CG_THREADS) v += __ldcg(a.part + i);
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int i = 0; i < CG_WARPS; i++) s += w[i];
      a.tot[k & 1] = s;
      __threadfence();
      atomicExch(a.rel, k);
      flag = 1;
    }
  } else if (threadIdx.x == 0) {
    // poll with a growing pause: hundreds of CTAs reading one L2 line at full
    // rate would queue the arrivals and the release behind the polls
    int good = 0;
    unsigned pause = 32;
    for (unsigned i = 0; i < CG_SPIN; i++) {
      if (ld_acquire(a.rel) >= k) {
        good = 1;
        break;
      }
      if (*(volatile int*)&a.status[ST_ERR]) break;
      __nanosleep(pause);
      if (pause < 128) pause <<= 1;
    }
    if (!good) set_err(a, ERR_TIMEOUT);
    __threadfence();
    flag = good;
  }
  __syncthreads();
  const int ok = flag;
  *total = __ldcg(a.tot + (k & 1));
  __syncthreads();  // flag and w are reused by the next call
  return ok;
}

// Row (x, j) of A v with v = u + beta w gathered at the neighbours (w may be
// null when beta is not used).  Result valid in every lane.  NB > 0 fixes
// nb at compile time (one k per lane for NB = 32) so that the 9 direction
// loads are independent and all in flight together.
template <int NB>
__device__ __forceinline__ float2 row_apply(const CoarseCGArgs& a, int x, int j, const float2* u, const float2* w,
                                            float beta) {
  const int lane = threadIdx.x & 31;
  const int nb = NB > 0 ? NB : a.nb;
  float re = 0.f, im = 0.f;
#pragma unroll
  for (int d = 0; d < 9; d++) {
    const int y = dwfmg::coarse_nbr(a.Lc, x, d);
    const float2* Ar = a.A + (((size_t)x * 9 + d) * nb + j) * nb;
    const float2* uy = u + (size_t)y * nb;
    const float2* wy = w ? w + (size_t)y * nb : nullptr;
#pragma unroll
    for (int k0 = 0; k0 < (NB > 0 ? NB : 32); k0 += 32) {
      for (int k = k0 + lane; k < (NB > 0 ? k0 + 32 : nb); k += 32) {
        const float2 m = __ldg(Ar + k);
        float2 v = __ldcg(uy + k);
        if (wy) {
          const float2 q = __ldcg(wy + k);
          v.x = fmaf(beta, q.x, v.x);
          v.y = fmaf(beta, q.y, v.y);
        }
        re = fmaf(m.x, v.x, re);
        re = fmaf(-m.y, v.y, re);
        im = fmaf(m.x, v.y, im);
        im = fmaf(m.y, v.x, im);
      }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  return make_float2(re, im);
}

// Two rows at once (rows r0 and r0 + stride, the second only when valid):
// the loads of both are issued before either is reduced, doubling the bytes
// in flight per warp.
template <int NB>
__device__ __forceinline__ void row_apply2(const CoarseCGArgs& a, long long r0, long long r1, bool has1,
                                           const float2* u, const float2* w, float beta, float2& o0, float2& o1) {
  const int x0 = (int)(r0 / a.nb), j0 = (int)(r0 % a.nb);
  const int x1 = has1 ? (int)(r1 / a.nb) : x0, j1 = has1 ? (int)(r1 % a.nb) : j0;
  if (NB != 32) {  // generic width: one row after the other
    o0 = row_apply<NB>(a, x0, j0, u, w, beta);
    o1 = has1 ? row_apply<NB>(a, x1, j1, u, w, beta) : make_float2(0.f, 0.f);
    return;
  }
  const int lane = threadIdx.x & 31;
  float re0 = 0.f, im0 = 0.f, re1 = 0.f, im1 = 0.f;
#pragma unroll
  for (int d = 0; d < 9; d++) {
    const int y0 = dwfmg::coarse_nbr(a.Lc, x0, d), y1 = dwfmg::coarse_nbr(a.Lc, x1, d);
    const float2 m0 = __ldg(a.A + (((size_t)x0 * 9 + d) * 32 + j0) * 32 + lane);
    const float2 m1 = __ldg(a.A + (((size_t)x1 * 9 + d) * 32 + j1) * 32 + lane);
    float2 v0 = __ldcg(u + (size_t)y0 * 32 + lane), v1 = __ldcg(u + (size_t)y1 * 32 + lane);
    if (w) {
      const float2 q0 = __ldcg(w + (size_t)y0 * 32 + lane), q1 = __ldcg(w + (size_t)y1 * 32 + lane);
      v0.x = fmaf(beta, q0.x, v0.x);
      v0.y = fmaf(beta, q0.y, v0.y);
      v1.x = fmaf(beta, q1.x, v1.x);
      v1.y = fmaf(beta, q1.y, v1.y);
    }
    re0 = fmaf(m0.x, v0.x, re0);
    re0 = fmaf(-m0.y, v0.y, re0);
    im0 = fmaf(m0.x, v0.y, im0);
    im0 = fmaf(m0.y, v0.x, im0);
    re1 = fmaf(m1.x, v1.x, re1);
    re1 = fmaf(-m1.y, v1.y, re1);
    im1 = fmaf(m1.x, v1.y, im1);
    im1 = fmaf(m1.y, v1.x, im1);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    re0 += __shfl_xor_sync(0xffffffffu, re0, o);
    im0 += __shfl_xor_sync(0xffffffffu, im0, o);
    re1 += __shfl_xor_sync(0xffffffffu, re1, o);
    im1 += __shfl_xor_sync(0xffffffffu, im1, o);
  }
  o0 = make_float2(re0, im0);
  o1 = make_float2(re1, im1);
}

template <int NB>
__global__ void __launch_bounds__(CG_THREADS) k_coarse_cg(CoarseCGArgs a) {
  const int lane = threadIdx.x & 31;
  const long long warp = (long long)blockIdx.x * CG_WARPS + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * CG_WARPS;
  const long long rows = (long long)a.nc * a.nb;
  unsigned nbar = 0;
  // Each warp owns rows warp, warp + nwarps, warp + 2 nwarps, ... and takes
  // them two at a time.  body(row, value) is run by lane 0 for each row.
  auto sweep = [&](const float2* u, const float2* w, float beta, auto&& body) {
    for (long long r0 = warp; r0 < rows; r0 += 2 * nwarps) {
      const long long r1 = r0 + nwarps;
      const bool has1 = r1 < rows;
      float2 o0, o1;
      row_apply2<NB>(a, r0, r1, has1, u, w, beta, o0, o1);
      if (lane == 0) {
        body(r0, o0);
        if (has1) body(r1, o1);
      }
    }
  };

  // b = A rhs; r = b; both p buffers zero; e = 0.
  double acc = 0;
  sweep(a.rhs, nullptr, 0.f, [&](long long row, float2 b) {
    a.r[row] = b;
    a.p0[row] = make_float2(0.f, 0.f);
    a.p1[row] = make_float2(0.f, 0.f);
    a.e[row] = make_float2(0.f, 0.f);
    acc += (double)b.x * b.x + (double)b.y * b.y;
  });
  double bb;
  if (!reduce_barrier(a, ++nbar, acc, &bb)) return;
  if (!(bb > 0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.status[ST_ITERS] = 0;
      if (!isfinite(bb)) set_err(a, ERR_NAN);
    }
    return;
  }
  double rr = bb, beta = 0;
  int it = 0;
  while (it < a.maxiter) {
    it++;
    float2* pcur = (it & 1) ? a.p1 : a.p0;
    const float2* pprev = (it & 1) ? a.p0 : a.p1;
    // phase A: p_i = r + beta p_{i-1}; t = A p_i
    acc = 0;
    sweep(a.r, pprev, (float)beta, [&](long long row, float2 tv) {
      const float2 rv = __ldcg(a.r + row), pv = __ldcg(pprev + row);
      pcur[row] = make_float2(fmaf((float)beta, pv.x, rv.x), fmaf((float)beta, pv.y, rv.y));
      a.t[row] = tv;
      acc += (double)tv.x * tv.x + (double)tv.y * tv.y;
    });
    double pap;
    if (!reduce_barrier(a, ++nbar, acc, &pap)) return;
    if (!(pap > 0)) {  // A p = 0 with p != 0 cannot happen for a nonsingular A
      if (blockIdx.x == 0 && threadIdx.x == 0) set_err(a, ERR_NAN);
      return;
    }
    const double alpha = rr / pap;
    // phase B: q = A t; e += alpha p_i; r -= alpha q
    acc = 0;
    sweep(a.t, nullptr, 0.f, [&](long long row, float2 q) {
      const float2 pv = __ldcg(pcur + row);
      float2 ev = __ldcg(a.e + row), rv = __ldcg(a.r + row);
      ev.x = fmaf((float)alpha, pv.x, ev.x);
      ev.y = fmaf((float)alpha, pv.y, ev.y);
      rv.x = fmaf(-(float)alpha, q.x, rv.x);
      rv.y = fmaf(-(float)alpha, q.y, rv.y);
      a.e[row] = ev;
      a.r[row] = rv;
      acc += (double)rv.x * rv.x + (double)rv.y * rv.y;
    });
    double rrn;
    if (!reduce_barrier(a, ++nbar, acc, &rrn)) return;
    if (!isfinite(rrn)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_err(a, ERR_NAN);
      return;
    }
    beta = rrn / rr;
    rr = rrn;
    if (rr <= a.tol2 * bb) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.status[ST_ITERS] = it;
    if (a.acc) atomicAdd(&a.acc[0], it);
  }
}

}  // namespace

// e = (A^2)^-1 A rhs on one right-hand side, FP32 vectors [nc][nb].  Work
// buffers: r, p0, p1, t (each nc*nb float2), part (2 totals + one partial per
// CTA, doubles), and in dev_small (CG_SMALL_BYTES) the int[2] status and,
// each in a 128-byte line of its own, the arrival and release counters of
// the grid barrier.
// With acc == nullptr the call synchronises and returns the iteration count
// and any error; with acc set it only enqueues (no host synchronisation, so
// it can be captured in a CUDA graph) and the kernel adds its iteration count
// to acc[0] and ORs its error code into acc[1] for the caller to read later.
int coarse_cg_persistent(dwf_ctx* c, float2* e, const float2* rhs, const float2* A, const int Lc[4], int nc,
                         int nb, double tol, int maxiter, float2* work, double* part, int part_cap,
                         int* dev_small, int* acc, int* iters, cudaStream_t st) {
  // NB = 32 and 64 compiled with fixed nb (fully unrolled loads); others generic
  void (*kern)(CoarseCGArgs) = nb == 32 ? k_coarse_cg<32> : nb == 64 ? k_coarse_cg<64> : k_coarse_cg<0>;
  const int ki = nb == 32 ? 0 : nb == 64 ? 1 : 2;
  static int grid_cache[64][3];
  int dev = 0;
  DWF_CUDA(c, cudaGetDevice(&dev));
  int grid = (dev >= 0 && dev < 64) ? grid_cache[dev][ki] : 0;
  if (grid <= 0) {
    int nsm = 0, per = 0;
    DWF_CUDA(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    DWF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, CG_THREADS, 0));
    if (per < 1) return dwf_fail(c, DWF_ECUDA, "coarse CG kernel cannot be resident");
    grid = nsm * (per < 4 ? per : 4);
    if (dev >= 0 && dev < 64) grid_cache[dev][ki] = grid;
  }
  const long long rows = (long long)nc * nb;
  const long long need = (rows + CG_WARPS - 1) / CG_WARPS;
  if (grid > need) grid = (int)need;
  if (grid < 1) grid = 1;
  if (grid + 2 > part_cap) return dwf_fail(c, DWF_EINVAL, "coarse CG partial buffer too small");
  CoarseCGArgs a;
  a.A = A;
  for (int m = 0; m < 4; m++) a.Lc[m] = Lc[m];
  a.nc = nc;
  a.nb = nb;
  a.rhs = rhs;
  a.e = e;
  a.r = work;
  a.p0 = work + rows;
  a.p1 = work + 2 * rows;
  a.t = work + 3 * rows;
  a.part = part + 2;  // part[0..1]: the two grid totals
  a.tot = part;
  a.status = dev_small;
  a.bar = (unsigned*)(dev_small + 32);
  a.rel = (unsigned*)(dev_small + 64);
  a.acc = acc;
  a.tol2 = tol * tol;
  a.maxiter = maxiter;
  DWF_CUDA(c, cudaMemsetAsync(dev_small, 0, CG_SMALL_BYTES, st));
  void* args[] = {&a};
  c->launches++;
  DWF_CUDA(c, cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(CG_THREADS), args, 0, st));
  if (acc) {
    *iters = 0;
    return DWF_OK;
  }
  int hs[2] = {0, 0};
  DWF_CUDA(c, cudaMemcpyAsync(hs, dev_small, sizeof(hs), cudaMemcpyDeviceToHost, st));
  DWF_CUDA(c, cudaStreamSynchronize(st));
  *iters = hs[ST_ITERS];
  if (hs[ST_ERR] == ERR_TIMEOUT) return dwf_fail(c, DWF_ETIMEOUT, "coarse CG grid barrier timed out");
  if (hs[ST_ERR] == ERR_NAN) return dwf_fail(c, DWF_ENAN, "NaN in coarse solve");
  return DWF_OK;
}
