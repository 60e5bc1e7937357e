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
  double* part;        // [3][nblk] partial sums
  unsigned* bar;       // barrier counter, zero at launch
  int* status;         // [ST_ITERS], [ST_ERR]
  double tol2;
  int maxiter;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier number k (k = 1, 2, ...): returns false when the wait ran out
// or another CTA has already given up.
__device__ bool grid_barrier(const CoarseCGArgs& a, unsigned k) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(a.bar, 1u);
    const unsigned target = k * gridDim.x;
    int good = 0;
    for (unsigned i = 0; i < CG_SPIN; i++) {
      if (ld_acquire(a.bar) >= target) {
        good = 1;
        break;
      }
      if (*(volatile int*)&a.status[ST_ERR]) break;
      __nanosleep(32);
    }
    if (!good) atomicCAS(&a.status[ST_ERR], 0, ERR_TIMEOUT);
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of the nblk partials of one slot, same order in every CTA.
__device__ double total(const CoarseCGArgs& a, int slot) {
  __shared__ double s;
  if (threadIdx.x < 32) {
    double v = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) v += __ldcg(a.part + (size_t)slot * gridDim.x + i);
    v = warp_sum(v);
    if (threadIdx.x == 0) s = v;
  }
  __syncthreads();
  const double out = s;
  __syncthreads();
  return out;
}

// CTA-wide sum of one double per warp (lane 0 holds it) into part[slot][blockIdx].
__device__ void store_partial(const CoarseCGArgs& a, int slot, double v) {
  __shared__ double w[CG_WARPS];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < CG_WARPS; i++) s += w[i];
    a.part[(size_t)slot * gridDim.x + blockIdx.x] = s;
  }
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

template <int NB>
__global__ void __launch_bounds__(CG_THREADS) k_coarse_cg(CoarseCGArgs a) {
  const int lane = threadIdx.x & 31;
  const long long warp = (long long)blockIdx.x * CG_WARPS + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * CG_WARPS;
  const long long rows = (long long)a.nc * a.nb;
  unsigned nbar = 0;

  // b = A rhs; r = b; both p buffers zero; e = 0.
  double acc = 0;
  for (long long row = warp; row < rows; row += nwarps) {
    const int x = (int)(row / a.nb), j = (int)(row % a.nb);
    const float2 b = row_apply<NB>(a, x, j, a.rhs, nullptr, 0.f);
    if (lane == 0) {
      a.r[row] = b;
      a.p0[row] = make_float2(0.f, 0.f);
      a.p1[row] = make_float2(0.f, 0.f);
      a.e[row] = make_float2(0.f, 0.f);
      acc += (double)b.x * b.x + (double)b.y * b.y;
    }
  }
  store_partial(a, 0, acc);
  if (!grid_barrier(a, ++nbar)) return;
  const double bb = total(a, 0);
  if (!(bb > 0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.status[ST_ITERS] = 0;
      if (!isfinite(bb)) atomicCAS(&a.status[ST_ERR], 0, ERR_NAN);
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
    for (long long row = warp; row < rows; row += nwarps) {
      const int x = (int)(row / a.nb), j = (int)(row % a.nb);
      const float2 tv = row_apply<NB>(a, x, j, a.r, pprev, (float)beta);
      if (lane == 0) {
        const float2 rv = __ldcg(a.r + row), pv = __ldcg(pprev + row);
        pcur[row] = make_float2(fmaf((float)beta, pv.x, rv.x), fmaf((float)beta, pv.y, rv.y));
        a.t[row] = tv;
        acc += (double)tv.x * tv.x + (double)tv.y * tv.y;
      }
    }
    store_partial(a, 1, acc);
    if (!grid_barrier(a, ++nbar)) return;
    const double pap = total(a, 1);
    if (!(pap > 0)) {  // A p = 0 with p != 0 cannot happen for a nonsingular A
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&a.status[ST_ERR], 0, ERR_NAN);
      return;
    }
    const double alpha = rr / pap;
    // phase B: q = A t; e += alpha p_i; r -= alpha q
    acc = 0;
    for (long long row = warp; row < rows; row += nwarps) {
      const int x = (int)(row / a.nb), j = (int)(row % a.nb);
      const float2 q = row_apply<NB>(a, x, j, a.t, nullptr, 0.f);
      if (lane == 0) {
        const float2 pv = __ldcg(pcur + row);
        float2 ev = __ldcg(a.e + row), rv = __ldcg(a.r + row);
        ev.x = fmaf((float)alpha, pv.x, ev.x);
        ev.y = fmaf((float)alpha, pv.y, ev.y);
        rv.x = fmaf(-(float)alpha, q.x, rv.x);
        rv.y = fmaf(-(float)alpha, q.y, rv.y);
        a.e[row] = ev;
        a.r[row] = rv;
        acc += (double)rv.x * rv.x + (double)rv.y * rv.y;
      }
    }
    store_partial(a, 2, acc);
    if (!grid_barrier(a, ++nbar)) return;
    const double rrn = total(a, 2);
    if (!isfinite(rrn)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&a.status[ST_ERR], 0, ERR_NAN);
      return;
    }
    beta = rrn / rr;
    rr = rrn;
    if (rr <= a.tol2 * bb) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.status[ST_ITERS] = it;
}

}  // namespace

// e = (A^2)^-1 A rhs on one right-hand side, FP32 vectors [nc][nb].  Work
// buffers: r, p0, p1, t (each nc*nb float2), partials (3*grid doubles), and
// an int[2] status plus an unsigned barrier counter in dev_small (16 bytes).
int coarse_cg_persistent(dwf_ctx* c, float2* e, const float2* rhs, const float2* A, const int Lc[4], int nc,
                         int nb, double tol, int maxiter, float2* work, double* part, int part_cap,
                         int* dev_small, int* iters, cudaStream_t st) {
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
  if (3 * grid > part_cap) return dwf_fail(c, DWF_EINVAL, "coarse CG partial buffer too small");
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
  a.part = part;
  a.status = dev_small;
  a.bar = (unsigned*)(dev_small + 2);
  a.tol2 = tol * tol;
  a.maxiter = maxiter;
  DWF_CUDA(c, cudaMemsetAsync(dev_small, 0, 4 * sizeof(int), st));
  void* args[] = {&a};
  c->launches++;
  DWF_CUDA(c, cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(CG_THREADS), args, 0, st));
  int hs[2] = {0, 0};
  DWF_CUDA(c, cudaMemcpyAsync(hs, dev_small, sizeof(hs), cudaMemcpyDeviceToHost, st));
  DWF_CUDA(c, cudaStreamSynchronize(st));
  *iters = hs[ST_ITERS];
  if (hs[ST_ERR] == ERR_TIMEOUT) return dwf_fail(c, DWF_ETIMEOUT, "coarse CG grid barrier timed out");
  if (hs[ST_ERR] == ERR_NAN) return dwf_fail(c, DWF_ENAN, "NaN in coarse solve");
  return DWF_OK;
}
