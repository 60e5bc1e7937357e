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
  const float2* x0;    // optional initial guess (plain CG only): e = x0, r = A rhs - A^2 x0
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

  // b = A rhs; r = b; both p buffers zero; e = 0 (with an initial guess x0,
  // also t = A x0, then r = b - A t and e = x0; the tolerance stays relative
  // to |b|, the residual of the zero start)
  double acc = 0;
  sweep(a.rhs, nullptr, 0.f, [&](long long row, float2 b) {
    a.r[row] = b;
    a.p0[row] = make_float2(0.f, 0.f);
    a.p1[row] = make_float2(0.f, 0.f);
    a.e[row] = make_float2(0.f, 0.f);
    acc += (double)b.x * b.x + (double)b.y * b.y;
  });
  if (a.x0) sweep(a.x0, nullptr, 0.f, [&](long long row, float2 v) { a.t[row] = v; });
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
  if (a.x0) {
    acc = 0;
    sweep(a.t, nullptr, 0.f, [&](long long row, float2 q) {  // rows are owned by the same lane in every sweep
      float2 rv = a.r[row];
      rv.x -= q.x;
      rv.y -= q.y;
      a.r[row] = rv;
      a.e[row] = __ldcg(a.x0 + row);
      acc += (double)rv.x * rv.x + (double)rv.y * rv.y;
    });
    if (!reduce_barrier(a, ++nbar, acc, &rr)) return;
  }
  int it = 0;
  while (it < a.maxiter && !(a.x0 && rr <= a.tol2 * bb)) {
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
                         int* dev_small, int* acc, int* iters, cudaStream_t st, const float2* x0) {
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
  a.x0 = x0;
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

// ====================================================================== red-black coarse CG
// Red-black solve of A e = r on the coarse lattice (Sec. 5.3: the red-black
// coarse solver of the physical-point runs).  With even coarse extents the
// 9-point stencil couples each coarse site to itself and to sites of the other
// parity only, so with the even Schur complement S = A_ee - A_eo A_oo^-1 A_oe
// (hermitian when A is):
//   r'_e = r_e - A_eo A_oo^-1 r_o,   S^2 e_e = S r'_e (CG),
//   e_o = A_oo^-1 (r_o - A_oe e_e).
// Storage: Arb[x][9][nb][nb] with, for even x, the stencil A_d(x) unchanged and,
// for odd x, Arb[x][0] = A_0(x)^-1 and Arb[x][d] = A_0(x)^-1 A_d(x) (d = 1..8),
// formed once per operator in FP64 (k_rb_prepare).  Then S v = A_0 v -
// sum_d A_d u(x+d) on even x with u(y) = sum_d' Arb[y][d'] v(y+d') on odd y:
// two sweeps per application, the same bytes as one stencil apply.

namespace {

// Site of the h-th coarse site of parity par (extents even): coarse sites are
// lexicographic x + Lc0 (y + Lc1 (z + Lc2 t)); within an x-row the sites of
// one parity are every other one.
__device__ __forceinline__ int rb_site(const int Lc[4], int h, int par) {
  const int hx = Lc[0] >> 1;
  int r = h / hx;
  const int xh = h - r * hx;
  const int y = r % Lc[1];
  r /= Lc[1];
  const int z = r % Lc[2];
  const int t = r / Lc[2];
  const int x = 2 * xh + ((y + z + t + par) & 1);
  return x + Lc[0] * (y + Lc[1] * (z + Lc[2] * t));
}

// One CTA per coarse site.  Odd sites: Gauss-Jordan inverse of A_0(x) with
// partial pivoting in FP64 (A_0 is hermitian but indefinite), then
// Arb[x][0] = A_0^-1 and Arb[x][d] = A_0^-1 A_d(x); even sites copy A_d(x).
// Dynamic shared memory: nb x 2nb complex FP64.  *fail is set when a pivot
// vanishes (a singular self block).
__global__ void __launch_bounds__(256) k_rb_prepare(const double2* __restrict__ A64, float2* __restrict__ Arb, int nb,
                                                    int Lc0, int Lc1, int Lc2, int Lc3, int* fail) {
  extern __shared__ double2 M[];  // row i: M[i * 2nb + j]
  __shared__ double fac_re[64], fac_im[64];
  __shared__ int piv;
  __shared__ double pmag;
  const int x = blockIdx.x;
  const int nn = nb * nb;
  int r = x;
  const int cx = r % Lc0;
  r /= Lc0;
  const int cy = r % Lc1;
  r /= Lc1;
  const int cz = r % Lc2;
  const int ct = r / Lc2;
  const double2* Ax = A64 + (size_t)x * 9 * nn;
  float2* Ox = Arb + (size_t)x * 9 * nn;
  if (((cx + cy + cz + ct) & 1) == 0) {
    for (int i = threadIdx.x; i < 9 * nn; i += blockDim.x) Ox[i] = make_float2((float)Ax[i].x, (float)Ax[i].y);
    return;
  }
  const int w2 = 2 * nb;
  for (int i = threadIdx.x; i < nb * w2; i += blockDim.x) {
    const int row = i / w2, col = i - row * w2;
    M[i] = col < nb ? Ax[row * nb + col] : make_double2(col - nb == row ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < nb; k++) {
    if (threadIdx.x < 32) {  // pivot: largest |M[i][k]| over i >= k
      double best = -1.0;
      int bi = k;
      for (int i = k + (int)threadIdx.x; i < nb; i += 32) {
        const double2 v = M[i * w2 + k];
        const double m = v.x * v.x + v.y * v.y;
        if (m > best) {
          best = m;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) {
        piv = bi;
        pmag = best;
      }
    }
    __syncthreads();
    if (!(pmag > 1e-280)) {
      if (threadIdx.x == 0) atomicExch(fail, 1);
      return;  // uniform: every thread read the same pmag
    }
    const int p = piv;
    if (p != k)
      for (int j = threadIdx.x; j < w2; j += blockDim.x) {
        const double2 a = M[k * w2 + j];
        M[k * w2 + j] = M[p * w2 + j];
        M[p * w2 + j] = a;
      }
    __syncthreads();
    const double2 d = M[k * w2 + k];
    const double den = d.x * d.x + d.y * d.y;
    const double ir = d.x / den, ii = -d.y / den;  // 1 / d
    __syncthreads();  // every thread has read the pivot
    for (int j = threadIdx.x; j < w2; j += blockDim.x) {
      const double2 a = M[k * w2 + j];
      M[k * w2 + j] = make_double2(a.x * ir - a.y * ii, a.x * ii + a.y * ir);
    }
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
      fac_re[i] = M[i * w2 + k].x;
      fac_im[i] = M[i * w2 + k].y;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nb * w2; e += blockDim.x) {
      const int i = e / w2, j = e - i * w2;
      if (i == k) continue;
      const double fr = fac_re[i], fi = fac_im[i];
      const double2 kj = M[k * w2 + j];
      double2 v = M[e];
      v.x -= fr * kj.x - fi * kj.y;
      v.y -= fr * kj.y + fi * kj.x;
      M[e] = v;
    }
    __syncthreads();
  }
  // A_0^-1 is the right half; store it, then stage each A_d in the left half
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int i = e / nb, j = e - i * nb;
    const double2 v = M[i * w2 + nb + j];
    Ox[e] = make_float2((float)v.x, (float)v.y);
  }
  for (int d = 1; d < 9; d++) {
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = e / nb, j = e - i * nb;
      M[i * w2 + j] = Ax[(size_t)d * nn + e];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = e / nb, j = e - i * nb;
      double re = 0.0, im = 0.0;
      for (int l = 0; l < nb; l++) {
        const double2 a = M[i * w2 + nb + l], b = M[l * w2 + j];
        re += a.x * b.x - a.y * b.y;
        im += a.x * b.y + a.y * b.x;
      }
      Ox[(size_t)d * nn + e] = make_float2((float)re, (float)im);
    }
  }
}

struct RBArgs {
  CoarseCGArgs a;   // A = Arb; r, p0, p1, t on even sites; e on all sites
  float2* u;        // odd-site intermediate
  float2* w;        // odd-site A_oo^-1 r_o (kept for the reconstruction)
  float2* rp;       // even-site r'_e
};

// Row (x, j) of  s0 * sum_{d in [d0, d1)} Arb[x][d][j][:] . v(x + d), v = u
// (+ beta w) gathered at the neighbours; result in every lane.
template <int NB>
__device__ __forceinline__ float2 rb_row(const CoarseCGArgs& a, int x, int j, int d0, int d1, const float2* u,
                                         const float2* w, float beta) {
  const int lane = threadIdx.x & 31;
  const int nb = NB > 0 ? NB : a.nb;
  float re = 0.f, im = 0.f;
  for (int d = d0; d < d1; d++) {
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
__global__ void __launch_bounds__(CG_THREADS) k_coarse_rbcg(RBArgs ra) {
  const CoarseCGArgs& a = ra.a;
  const int lane = threadIdx.x & 31;
  const long long warp = (long long)blockIdx.x * CG_WARPS + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * CG_WARPS;
  const long long rows = (long long)(a.nc / 2) * a.nb;  // rows of one parity
  unsigned nbar = 0;
  // body(site, j, row index) for every row of parity par, run by lane 0
  auto sweep = [&](int par, auto&& rowfn, auto&& body) {
    for (long long rr = warp; rr < rows; rr += nwarps) {
      const int h = (int)(rr / a.nb), j = (int)(rr % a.nb);
      const int x = rb_site(a.Lc, h, par);
      const float2 v = rowfn(x, j);
      if (lane == 0) body((long long)x * a.nb + j, v);
    }
  };
  auto bar = [&]() -> bool {
    double dummy;
    return reduce_barrier(a, ++nbar, 0.0, &dummy);
  };
  // prologue: w_o = A_oo^-1 r_o; r'_e = r_e - A_eo w_o; u_o = (A_oo^-1 A_oe) r'_e;
  // b = A_ee r'_e - A_eo u_o; r = b; e = p = 0
  sweep(1, [&](int x, int j) { return rb_row<NB>(a, x, j, 0, 1, a.rhs, nullptr, 0.f); },
        [&](long long row, float2 v) { ra.w[row] = v; });
  if (!bar()) return;
  sweep(0, [&](int x, int j) { return rb_row<NB>(a, x, j, 1, 9, ra.w, nullptr, 0.f); },
        [&](long long row, float2 v) {
          const float2 rv = __ldcg(a.rhs + row);
          ra.rp[row] = make_float2(rv.x - v.x, rv.y - v.y);
        });
  if (!bar()) return;
  sweep(1, [&](int x, int j) { return rb_row<NB>(a, x, j, 1, 9, ra.rp, nullptr, 0.f); },
        [&](long long row, float2 v) { ra.u[row] = v; });
  if (!bar()) return;
  double acc = 0;
  sweep(0, [&](int x, int j) {
          const float2 s0 = rb_row<NB>(a, x, j, 0, 1, ra.rp, nullptr, 0.f);
          const float2 s1 = rb_row<NB>(a, x, j, 1, 9, ra.u, nullptr, 0.f);
          return make_float2(s0.x - s1.x, s0.y - s1.y);
        },
        [&](long long row, float2 b) {
          a.r[row] = b;
          a.p0[row] = make_float2(0.f, 0.f);
          a.p1[row] = make_float2(0.f, 0.f);
          a.e[row] = make_float2(0.f, 0.f);
          acc += (double)b.x * b.x + (double)b.y * b.y;
        });
  double bb;
  if (!reduce_barrier(a, ++nbar, acc, &bb)) return;
  int it = 0;
  if (bb > 0) {
    double rr = bb, beta = 0;
    while (it < a.maxiter) {
      it++;
      float2* pcur = (it & 1) ? a.p1 : a.p0;
      const float2* pprev = (it & 1) ? a.p0 : a.p1;
      // t = S p, p = r + beta p_prev formed where it is read
      sweep(1, [&](int x, int j) { return rb_row<NB>(a, x, j, 1, 9, a.r, pprev, (float)beta); },
            [&](long long row, float2 v) { ra.u[row] = v; });
      if (!bar()) return;
      acc = 0;
      sweep(0, [&](int x, int j) {
              const float2 s0 = rb_row<NB>(a, x, j, 0, 1, a.r, pprev, (float)beta);
              const float2 s1 = rb_row<NB>(a, x, j, 1, 9, ra.u, nullptr, 0.f);
              return make_float2(s0.x - s1.x, s0.y - s1.y);
            },
            [&](long long row, float2 tv) {
              const float2 rv = __ldcg(a.r + row), pv = __ldcg(pprev + row);
              pcur[row] = make_float2(fmaf((float)beta, pv.x, rv.x), fmaf((float)beta, pv.y, rv.y));
              a.t[row] = tv;
              acc += (double)tv.x * tv.x + (double)tv.y * tv.y;
            });
      double pap;
      if (!reduce_barrier(a, ++nbar, acc, &pap)) return;
      if (!(pap > 0)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_err(a, ERR_NAN);
        return;
      }
      const double alpha = rr / pap;
      // q = S t; e += alpha p; r -= alpha q
      sweep(1, [&](int x, int j) { return rb_row<NB>(a, x, j, 1, 9, a.t, nullptr, 0.f); },
            [&](long long row, float2 v) { ra.u[row] = v; });
      if (!bar()) return;
      acc = 0;
      sweep(0, [&](int x, int j) {
              const float2 s0 = rb_row<NB>(a, x, j, 0, 1, a.t, nullptr, 0.f);
              const float2 s1 = rb_row<NB>(a, x, j, 1, 9, ra.u, nullptr, 0.f);
              return make_float2(s0.x - s1.x, s0.y - s1.y);
            },
            [&](long long row, float2 q) {
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
  } else if (!isfinite(bb)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_err(a, ERR_NAN);
    return;
  } else {  // r'_e = 0: e_e = 0
    sweep(0, [&](int x, int j) { return make_float2(0.f, 0.f); },
          [&](long long row, float2) { a.e[row] = make_float2(0.f, 0.f); });
    if (!bar()) return;
  }
  // e_o = w_o - (A_oo^-1 A_oe) e_e
  sweep(1, [&](int x, int j) { return rb_row<NB>(a, x, j, 1, 9, a.e, nullptr, 0.f); },
        [&](long long row, float2 v) {
          const float2 wv = __ldcg(ra.w + row);
          a.e[row] = make_float2(wv.x - v.x, wv.y - v.y);
        });
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.status[ST_ITERS] = it;
    if (a.acc) atomicAdd(&a.acc[0], it);
  }
}

}  // namespace

// Arb (see above) from the FP64 operator; DWF_ERANGE when an odd self block
// is singular.  Synchronises.
int coarse_rb_prepare(dwf_ctx* c, const double2* A64, float2* Arb, const int Lc[4], int nc, int nb, int* dev_flag,
                      cudaStream_t st) {
  const size_t smem = (size_t)nb * 2 * nb * sizeof(double2);
  static size_t opted = 48 * 1024;
  if (smem > opted) {
    DWF_CUDA(c, cudaFuncSetAttribute(k_rb_prepare, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    opted = smem;
  }
  DWF_CUDA(c, cudaMemsetAsync(dev_flag, 0, sizeof(int), st));
  c->launches++;
  k_rb_prepare<<<nc, 256, smem, st>>>(A64, Arb, nb, Lc[0], Lc[1], Lc[2], Lc[3], dev_flag);
  DWF_CUDA(c, cudaGetLastError());
  int h = 0;
  DWF_CUDA(c, cudaMemcpyAsync(&h, dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  DWF_CUDA(c, cudaStreamSynchronize(st));
  if (h) return dwf_fail(c, DWF_ERANGE, "red-black coarse solve: a self block of the coarse operator is singular");
  return DWF_OK;
}

// Red-black CG (above) for one right-hand side: e = A^-1 rhs by CG on S^2 to
// a relative normal residual tol.  work: 7 nc nb float2; other arguments as
// coarse_cg_persistent.
int coarse_rbcg_persistent(dwf_ctx* c, float2* e, const float2* rhs, const float2* Arb, const int Lc[4], int nc,
                           int nb, double tol, int maxiter, float2* work, double* part, int part_cap, int* dev_small,
                           int* acc, int* iters, cudaStream_t st) {
  for (int m = 0; m < 4; m++)
    if (Lc[m] & 1) return dwf_fail(c, DWF_EINVAL, "red-black coarse solve needs even coarse extents");
  if (nb > 64) return dwf_fail(c, DWF_EINVAL, "nb > 64");
  void (*kern)(RBArgs) = nb == 32 ? k_coarse_rbcg<32> : nb == 64 ? k_coarse_rbcg<64> : k_coarse_rbcg<0>;
  const int ki = nb == 32 ? 0 : nb == 64 ? 1 : 2;
  static int grid_cache[64][3];
  int dev = 0;
  DWF_CUDA(c, cudaGetDevice(&dev));
  int grid = (dev >= 0 && dev < 64) ? grid_cache[dev][ki] : 0;
  if (grid <= 0) {
    int nsm = 0, per = 0;
    DWF_CUDA(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    DWF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, CG_THREADS, 0));
    if (per < 1) return dwf_fail(c, DWF_ECUDA, "red-black coarse CG kernel cannot be resident");
    grid = nsm * (per < 4 ? per : 4);
    if (dev >= 0 && dev < 64) grid_cache[dev][ki] = grid;
  }
  const long long rows = (long long)(nc / 2) * nb;
  const long long need = (rows + CG_WARPS - 1) / CG_WARPS;
  if (grid > need) grid = (int)need;
  if (grid < 1) grid = 1;
  if (grid + 2 > part_cap) return dwf_fail(c, DWF_EINVAL, "coarse CG partial buffer too small");
  const long long n = (long long)nc * nb;
  RBArgs ra;
  CoarseCGArgs& a = ra.a;
  a.A = Arb;
  for (int m = 0; m < 4; m++) a.Lc[m] = Lc[m];
  a.nc = nc;
  a.nb = nb;
  a.rhs = rhs;
  a.e = e;
  a.r = work;
  a.p0 = work + n;
  a.p1 = work + 2 * n;
  a.t = work + 3 * n;
  ra.u = work + 4 * n;
  ra.w = work + 5 * n;
  ra.rp = work + 6 * n;
  a.part = part + 2;
  a.tot = part;
  a.status = dev_small;
  a.bar = (unsigned*)(dev_small + 32);
  a.rel = (unsigned*)(dev_small + 64);
  a.acc = acc;
  a.tol2 = tol * tol;
  a.maxiter = maxiter;
  a.x0 = nullptr;
  DWF_CUDA(c, cudaMemsetAsync(dev_small, 0, CG_SMALL_BYTES, st));
  void* args[] = {&ra};
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
