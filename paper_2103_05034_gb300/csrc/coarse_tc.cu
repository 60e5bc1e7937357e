// Coarse 9-point stencil on the 5th-generation tensor cores (tcgen05, TF32
// inputs, FP32 accumulation in tensor memory): out(x) = sum_d A_d(x) in(x+d)
// for many right-hand sides (Sec. 3.1, Eq. 18: the little Dirac operator is a
// dense nb x nb block stencil, a real dense contraction).
//
// Real form of one complex block product (nb = 32):
//   [Re out; Im out] (64 x N) = [[Ar, -Ai], [Ai, Ar]] (64 x 64) [Re in; Im in] (64 x N)
// tcgen05.mma with M = 128 takes two coarse sites at once: the A tile of one
// direction stacks site x1's 64 rows over site x2's (K = 64, no zero blocks),
// and two MMA chains multiply it by x1's and by x2's B block into two column
// ranges of the accumulator; rows 0-63 of the first range and rows 64-127 of
// the second are the two results (the other quadrants are discarded).  One
// pipeline stage per direction holds
//   A: [K/4 = 16][M = 128][4] TF32 (32 KB, one cp.async.bulk from a copy of
//      the operator pre-arranged per site pair)
//   B: 2 x [K/4 = 16][N][4] TF32 (2 x N*256 B, the neighbours' blocks of a
//      pre-arranged copy of the right-hand sides)
// in the canonical no-swizzle K-major layout (8-row x 16-byte core matrices;
// K-adjacent cores LBO apart, M/N-adjacent cores 128 B apart); 3 to 5 stages
// in flight, 16 MMAs of K = 8 per stage, one tcgen05.commit per stage.
#include <string.h>

#include "dwf_internal.cuh"
#include "mg_kernels.cuh"

namespace {

constexpr int TC_NB = 32;           // basis vectors per site handled here
constexpr int TC_ROWS = 2 * TC_NB;  // real rows per site
constexpr int TC_M = 128;
constexpr int TC_K = 64;            // per stage and site
constexpr int TC_THREADS = 128;     // epilogue warps; one more warp issues copies and MMAs
constexpr unsigned TC_SPIN = 1u << 22;  // bounded waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);  // version 1, no swizzle
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned i = 0; i < TC_SPIN; i++) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Pre-arranged operator, per pair of coarse sites (2p, 2p+1) and direction:
// At[p][d][kg = 16][r = 128][4] TF32 (real form, K-major), rows 0-63 site 2p
// and rows 64-127 site 2p+1, so that one stage's A tile is one contiguous
// 32 KB bulk copy.
__global__ void k_tc_arrange(float* At, const float2* A, int nc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (x, d, r, k)
  if (e >= (long long)nc * 9 * TC_ROWS * TC_ROWS) return;
  const int k = (int)(e % TC_ROWS);
  const int r = (int)((e / TC_ROWS) % TC_ROWS);
  const long long xd = e / (TC_ROWS * TC_ROWS);
  const long long x = xd / 9;
  const int d = (int)(xd % 9);
  const int j = r % TC_NB, kk = k % TC_NB;
  const float2 a = A[(xd * TC_NB + j) * TC_NB + kk];
  float v;
  if (r < TC_NB)
    v = k < TC_NB ? a.x : -a.y;
  else
    v = k < TC_NB ? a.y : a.x;
  const long long pd = (x >> 1) * 9 + d;
  const int row = (int)(x & 1) * TC_ROWS + r;
  At[((pd * (TC_ROWS / 4) + k / 4) * TC_M + row) * 4 + (k & 3)] = to_tf32(v);
}

// Pre-arranged right-hand sides: Bt[y][kg = 16][n = N][4] TF32, K index
// k < 32 the real part and k >= 32 the imaginary part of in[y][k mod 32][n]
// (the K-major no-swizzle layout of one site's 64 x N B block), so that the
// main kernel fetches a neighbour's block with one bulk copy.
__global__ void k_tc_arrange_in(float* Bt, const float2* in, int nc, int N) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (y, j, n)
  if (e >= (long long)nc * TC_NB * N) return;
  const int n = (int)(e % N);
  const int j = (int)((e / N) % TC_NB);
  const long long y = e / ((long long)N * TC_NB);
  const float2 v = in[e];
  const int kre = j, kim = TC_NB + j;
  Bt[((y * (TC_ROWS / 4) + kre / 4) * N + n) * 4 + (kre & 3)] = to_tf32(v.x);
  Bt[((y * (TC_ROWS / 4) + kim / 4) * N + n) * 4 + (kim & 3)] = to_tf32(v.y);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Pipeline depth for N right-hand sides: as many 32 KB + N*512 B stages as
// fit in about 220 KB of shared memory, at most 5.
template <int N>
struct TcStages {
  static constexpr int bytes = (TC_K / 4) * TC_M * 16 + 2 * (TC_K / 4) * N * 16;
  static constexpr int v = (220 * 1024 / bytes) < 5 ? (220 * 1024 / bytes) : 5;
};

// Persistent, warp-specialised coarse stencil.  Each CTA walks pairs of
// coarse sites (x1, x2) = (2p, 2p+1), p = blockIdx.x, blockIdx.x + gridDim.x,
// ...; one pair is 9 pipeline stages (one per stencil direction d).
//   warp 4 (one elected thread): for stage g, waits until the MMAs of stage
//     g-S have released shared-memory buffer g%S, posts the stage's bytes on
//     full[g%S] and issues its three bulk copies (A_d of the pair, 32 KB; the
//     neighbours' B blocks, 2 x N*256 B); then issues the 16 MMAs of stage
//     g-S+1 once its copies have landed and commits them to done[(g-S+1)%S]
//     (and, after a pair's last direction, to acc_full[t]).  S-1 stages of
//     copies are in flight while one stage multiplies.
//   warps 0-3: per pair, wait acc_full[t], read the accumulator (TMEM lane =
//     stacked row; rows 0-63 from the first column range, 64-127 from the
//     second) with tcgen05.ld, store it, and arrive on acc_empty[t]; the
//     producer waits on acc_empty[t] before the first MMA of the pair two
//     later, which reuses accumulator t (two accumulators of 2N columns in
//     TMEM, so a pair's epilogue overlaps the next pair's MMAs).
// Every wait is bounded; a thread whose wait runs out sets *err and stops
// issuing work, and the producer waits (bounded) for copies still in flight
// before the CTA frees its tensor memory.
template <int N>
__global__ void __launch_bounds__(TC_THREADS + 32, 1)
    k_coarse_apply_tc(float2* out, const float* Bt, const float* At, int Lc0, int Lc1, int Lc2, int Lc3,
                      int npairs, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int S = TcStages<N>::v;
  constexpr int A_BYTES = (TC_K / 4) * TC_M * 16;  // 32 KB
  constexpr int B_BYTES = (TC_K / 4) * N * 16;     // one site's block
  constexpr int ST_BYTES = A_BYTES + 2 * B_BYTES;
  constexpr uint32_t LBO_A = TC_M * 16, LBO_B = N * 16, SBO = 128;
  constexpr uint32_t NCOL = 2 * N;  // one accumulator: two column ranges of N
  constexpr uint32_t TCOLS = 2 * NCOL;
  static_assert(NCOL % 32 == 0 && (TCOLS & (TCOLS - 1)) == 0, "TMEM allocation is a power of two >= 32");
  uint64_t* bars = (uint64_t*)(smem + S * ST_BYTES);
  // bars: full[0..S), done[S..2S), acc_full[2S..2S+2), acc_empty[2S+2..2S+4)
  uint64_t* full = bars;
  uint64_t* done = bars + S;
  uint64_t* acc_full = bars + 2 * S;
  uint64_t* acc_empty = bars + 2 * S + 2;
  uint32_t* tslot = (uint32_t*)(bars + 2 * S + 4);
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Lc[4] = {Lc0, Lc1, Lc2, Lc3};

  if (tid == 0) {
    for (int i = 0; i < 2 * S + 2; i++) mbar_init(smem_u32(bars + i), 1);
    for (int i = 0; i < 2; i++) mbar_init(smem_u32(acc_empty + i), TC_THREADS);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
                             ((uint32_t)(TC_M >> 4) << 24);
  const int mypairs = (int)blockIdx.x < npairs ? (npairs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (warp == 4) {
    if (lane == 0) {
      bool ok = true;
      const int nst = mypairs * 9;
      int issued = 0;  // stages whose copies were issued
      auto mma_stage = [&](int h) -> bool {
        const int pl = h / 9, d = h % 9, t = pl & 1, b = h % S;
        if (d == 0 && pl >= 2 && !mbar_wait(smem_u32(acc_empty + t), ((pl - 2) >> 1) & 1)) return false;
        if (!mbar_wait(smem_u32(full + b), (h / S) & 1)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(smem + b * ST_BYTES);
#pragma unroll
        for (int q = 0; q < 2; q++) {  // site q's B block into column range q
          const uint32_t b0 = a0 + A_BYTES + q * B_BYTES;
#pragma unroll
          for (int kk = 0; kk < TC_K / 8; kk++) {
            const uint64_t ad = smem_desc(a0 + kk * 2 * LBO_A, LBO_A, SBO);
            const uint64_t bd = smem_desc(b0 + kk * 2 * LBO_B, LBO_B, SBO);
            const uint32_t acc = (d > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + t * NCOL + q * N),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
        }
        tc_commit(smem_u32(done + b));
        if (d == 8) tc_commit(smem_u32(acc_full + t));
        return true;
      };
      for (int g = 0; g < nst && ok; g++) {
        const int pl = g / 9, d = g % 9, b = g % S;
        const int p = blockIdx.x + pl * gridDim.x;
        if (g >= S && !mbar_wait(smem_u32(done + b), ((g - S) / S) & 1)) {
          ok = false;
          break;
        }
        unsigned char* st = smem + b * ST_BYTES;
        const uint32_t fb = smem_u32(full + b);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(ST_BYTES) : "memory");
        bulk_g2s(smem_u32(st), At + ((long long)p * 9 + d) * (TC_ROWS / 4) * TC_M * 4, A_BYTES, fb);
        for (int q = 0; q < 2; q++) {
          const int y = dwfmg::coarse_nbr(Lc, 2 * p + q, d);
          bulk_g2s(smem_u32(st + A_BYTES + q * B_BYTES), Bt + (long long)y * (TC_ROWS / 4) * N * 4, B_BYTES, fb);
        }
        issued = g + 1;
        if (g >= S - 1 && !mma_stage(g - (S - 1))) {
          ok = false;
          break;
        }
      }
      for (int h = (nst > S - 1 ? nst - (S - 1) : 0); ok && h < nst; h++)
        if (!mma_stage(h)) ok = false;
      if (!ok) {
        atomicExch(err, 1);
        atomicExch(&abort_flag, 1);
        // let copies still in flight land before the CTA exits (bounded)
        for (int h = (issued >= S ? issued - S : 0); h < issued; h++) mbar_wait(smem_u32(full + h % S), (h / S) & 1);
      }
    }
  } else {
    // epilogue warps 0-3: warp w owns TMEM lanes 32w..32w+31 = stacked rows;
    // rows 0-63 are site x1 (column range 0), rows 64-127 site x2 (range 1)
    const int r = warp * 32 + lane;
    const int q = r / TC_ROWS, rr = r % TC_ROWS;
    const int part = rr / TC_NB, j = rr % TC_NB;
    for (int pl = 0; pl < mypairs; pl++) {
      const int t = pl & 1;
      const int p = blockIdx.x + pl * gridDim.x;
      if (!mbar_wait(smem_u32(acc_full + t), (pl >> 1) & 1)) {
        atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* o = (float*)(out + ((long long)(2 * p + q) * TC_NB + j) * N) + part;
#pragma unroll
      for (int c0 = 0; c0 < N; c0 += 16) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + t * NCOL + q * N + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 16; i++) o[2 * (c0 + i)] = __uint_as_float(v[i]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acc_empty + t)) : "memory");
      if (*(volatile int*)&abort_flag) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
  }
}

// ---------------------------------------------------------------- complex-split form
// The same stencil with the operator kept complex: per site and direction
//   A' = [Re A | Im A]  (32 x 64),   B' = [[Re B, Im B], [-Im B, Re B]]  (64 x 2N),
//   A' B' = [Re(A B) | Im(A B)],
// so the operator streams at its complex FP32 size (half the real form's).
// One MMA tile (M = 128) stacks the A' of four consecutive coarse sites (a
// quad); site q's neighbour block B'_q goes through the whole tile into
// accumulator columns [q 2N, (q+1) 2N), whose rows 32q..32q+31 -- TMEM lanes
// of epilogue warp q -- are site q's result.  One stage per (quad, direction):
//   A: [K/4 = 16][M = 128][4] TF32, 32 KB, one bulk copy of the operator
//      pre-arranged per quad;
//   B: 4 x [K/4 = 16][2N][4] TF32 (N*512 B each), the neighbours' arranged blocks.
// Accumulator: 4 x 2N columns, double buffered (N <= 32).
__global__ void k_tc4_arrange(float* At, const float2* A, int nc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (x, d, j, k)
  if (e >= (long long)nc * 9 * TC_NB * TC_NB) return;
  const int k = (int)(e % TC_NB);
  const int j = (int)((e / TC_NB) % TC_NB);
  const long long xd = e / (TC_NB * TC_NB);
  const long long x = xd / 9;
  const int d = (int)(xd % 9);
  const float2 a = A[e];
  const long long qd = (x >> 2) * 9 + d;
  const int row = (int)(x & 3) * TC_NB + j;
  float* base = At + qd * (TC_ROWS / 4) * TC_M * 4;
  base[((k / 4) * TC_M + row) * 4 + (k & 3)] = to_tf32(a.x);                      // K index k: Re A
  base[(((TC_NB + k) / 4) * TC_M + row) * 4 + ((TC_NB + k) & 3)] = to_tf32(a.y);  // K index 32 + k: Im A
}

__global__ void k_tc4_arrange_in(float* Bt, const float2* in, int nc, int N) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (y, k, n)
  if (e >= (long long)nc * TC_NB * N) return;
  const int n = (int)(e % N);
  const int k = (int)((e / N) % TC_NB);
  const long long y = e / ((long long)N * TC_NB);
  const float2 v = in[e];
  const int N2 = 2 * N;
  float* base = Bt + y * (TC_ROWS / 4) * N2 * 4;
  auto put = [&](int kk, int nn, float val) { base[((kk / 4) * N2 + nn) * 4 + (kk & 3)] = to_tf32(val); };
  put(k, n, v.x);
  put(k, N + n, v.y);
  put(TC_NB + k, n, -v.y);
  put(TC_NB + k, N + n, v.x);
}

template <int N>
struct Tc4Stages {
  static constexpr int bytes = (TC_K / 4) * TC_M * 16 + 4 * (TC_K / 4) * (2 * N) * 16;
  static constexpr int v = (220 * 1024 / bytes) < 4 ? (220 * 1024 / bytes) : 4;
};

// Persistent, warp-specialised as k_coarse_apply_tc, over quads instead of
// pairs: warp 4 (one elected thread) issues each stage's five bulk copies and,
// S-1 stages behind, its 32 MMAs (4 sites x 8 K-steps); warps 0-3 drain the
// accumulator, warp q writing site q of the quad.  Bounded waits as there.
template <int N>
__global__ void __launch_bounds__(TC_THREADS + 32, 1)
    k_coarse_apply_tc4(float2* out, const float* Bt, const float* At, int Lc0, int Lc1, int Lc2, int Lc3,
                       int nquads, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int S = Tc4Stages<N>::v;
  constexpr int N2 = 2 * N;
  constexpr int A_BYTES = (TC_K / 4) * TC_M * 16;  // 32 KB
  constexpr int B_BYTES = (TC_K / 4) * N2 * 16;    // one site's B'
  constexpr int ST_BYTES = A_BYTES + 4 * B_BYTES;
  constexpr uint32_t LBO_A = TC_M * 16, LBO_B = N2 * 16, SBO = 128;
  constexpr uint32_t NCOL = 4 * N2;  // one accumulator: four column ranges of 2N
  constexpr uint32_t TCOLS = 2 * NCOL;
  static_assert(TCOLS <= 512 && (TCOLS & (TCOLS - 1)) == 0, "TMEM allocation is a power of two <= 512");
  static_assert(S >= 2, "at least two pipeline stages");
  uint64_t* bars = (uint64_t*)(smem + S * ST_BYTES);
  uint64_t* full = bars;
  uint64_t* done = bars + S;
  uint64_t* acc_full = bars + 2 * S;
  uint64_t* acc_empty = bars + 2 * S + 2;
  uint32_t* tslot = (uint32_t*)(bars + 2 * S + 4);
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Lc[4] = {Lc0, Lc1, Lc2, Lc3};

  if (tid == 0) {
    for (int i = 0; i < 2 * S + 2; i++) mbar_init(smem_u32(bars + i), 1);
    for (int i = 0; i < 2; i++) mbar_init(smem_u32(acc_empty + i), TC_THREADS);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N2 >> 3) << 17) |
                             ((uint32_t)(TC_M >> 4) << 24);
  const int myq = (int)blockIdx.x < nquads ? (nquads - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (warp == 4) {
    if (lane == 0) {
      bool ok = true;
      const int nst = myq * 9;
      int issued = 0;
      auto mma_stage = [&](int h) -> bool {
        const int ql = h / 9, d = h % 9, t = ql & 1, b = h % S;
        if (d == 0 && ql >= 2 && !mbar_wait(smem_u32(acc_empty + t), ((ql - 2) >> 1) & 1)) return false;
        if (!mbar_wait(smem_u32(full + b), (h / S) & 1)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(smem + b * ST_BYTES);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint32_t b0 = a0 + A_BYTES + q * B_BYTES;
#pragma unroll
          for (int kk = 0; kk < TC_K / 8; kk++) {
            const uint64_t ad = smem_desc(a0 + kk * 2 * LBO_A, LBO_A, SBO);
            const uint64_t bd = smem_desc(b0 + kk * 2 * LBO_B, LBO_B, SBO);
            const uint32_t acc = (d > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + t * NCOL + q * N2),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
          }
        }
        tc_commit(smem_u32(done + b));
        if (d == 8) tc_commit(smem_u32(acc_full + t));
        return true;
      };
      for (int g = 0; g < nst && ok; g++) {
        const int ql = g / 9, d = g % 9, b = g % S;
        const int qd = blockIdx.x + ql * gridDim.x;
        if (g >= S && !mbar_wait(smem_u32(done + b), ((g - S) / S) & 1)) {
          ok = false;
          break;
        }
        unsigned char* st = smem + b * ST_BYTES;
        const uint32_t fb = smem_u32(full + b);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(ST_BYTES) : "memory");
        bulk_g2s(smem_u32(st), At + ((long long)qd * 9 + d) * (TC_ROWS / 4) * TC_M * 4, A_BYTES, fb);
        for (int q = 0; q < 4; q++) {
          const int y = dwfmg::coarse_nbr(Lc, 4 * qd + q, d);
          bulk_g2s(smem_u32(st + A_BYTES + q * B_BYTES), Bt + (long long)y * (TC_ROWS / 4) * N2 * 4, B_BYTES, fb);
        }
        issued = g + 1;
        if (g >= S - 1 && !mma_stage(g - (S - 1))) {
          ok = false;
          break;
        }
      }
      for (int h = (nst > S - 1 ? nst - (S - 1) : 0); ok && h < nst; h++)
        if (!mma_stage(h)) ok = false;
      if (!ok) {
        atomicExch(err, 1);
        atomicExch(&abort_flag, 1);
        for (int h = (issued >= S ? issued - S : 0); h < issued; h++) mbar_wait(smem_u32(full + h % S), (h / S) & 1);
      }
    }
  } else {
    // epilogue: warp q owns TMEM lanes 32q..32q+31 = rows j of site 4 qd + q,
    // columns [q 2N, q 2N + N) the real parts and [q 2N + N, (q+1) 2N) the imaginary
    const int q = warp, j = lane;
    for (int ql = 0; ql < myq; ql++) {
      const int t = ql & 1;
      const int qd = blockIdx.x + ql * gridDim.x;
      if (!mbar_wait(smem_u32(acc_full + t), (ql >> 1) & 1)) {
        atomicExch(err, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* o = (float*)(out + ((long long)(4 * qd + q) * TC_NB + j) * N);
#pragma unroll
      for (int c0 = 0; c0 < N2; c0 += 16) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(tmem + t * NCOL + q * N2 + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int part = c0 < N ? 0 : 1, n0 = c0 < N ? c0 : c0 - N;
#pragma unroll
        for (int i = 0; i < 16; i++) o[2 * (n0 + i) + part] = __uint_as_float(v[i]);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acc_empty + t)) : "memory");
      if (*(volatile int*)&abort_flag) break;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
  }
}

}  // namespace

// Tensor-core coarse apply; returns DWF_EINVAL when the shape is not covered
// (nb != 32, an odd number of coarse sites, nrhs not 16, 32 or 64).  With a
// multiple of four coarse sites and nrhs <= 32 it runs the complex-split
// kernel (operator At4, built on first use), otherwise the real-form pair
// kernel (operator At); Bt (the arranged right-hand sides) is a buffer the
// coarse operator keeps, grown on demand.
int coarse_apply_tc(dwf_ctx* c, float2* out, const float2* in, const float2* A32, float** At, float** At4,
                    float** Bt, size_t* Bt_bytes, int nb, int nc, const int Lc[4], int nrhs, int* err_dev,
                    cudaStream_t st) {
  if (nb != TC_NB || (nc & 1) || (nrhs != 16 && nrhs != 32 && nrhs != 64)) return DWF_EINVAL;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm < 1) nsm = 1;
  }
  if ((nc & 3) == 0 && nrhs <= 32) {
    // complex-split form (quads of sites): the operator at its complex size
    if (!*At4) {
      if (cudaMalloc(At4, (size_t)nc * 9 * TC_NB * TC_ROWS * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return DWF_ENOMEM;
      }
      const long long n = (long long)nc * 9 * TC_NB * TC_NB;
      k_tc4_arrange<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(*At4, A32, nc);
      c->launches++;
    }
    const size_t bbytes = (size_t)nc * TC_ROWS * 2 * nrhs * sizeof(float);
    if (*Bt_bytes < bbytes) {
      if (*Bt) cudaFree(*Bt);
      *Bt = nullptr;
      *Bt_bytes = 0;
      if (cudaMalloc(Bt, bbytes) != cudaSuccess) {
        cudaGetLastError();
        return DWF_ENOMEM;
      }
      *Bt_bytes = bbytes;
    }
    const long long n = (long long)nc * TC_NB * nrhs;
    k_tc4_arrange_in<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(*Bt, in, nc, nrhs);
    c->launches += 2;
    const int nquads = nc / 4;
    const int grid = nquads < nsm ? nquads : nsm;
    int smem = 0;
    if (nrhs == 16) {
      smem = Tc4Stages<16>::v * Tc4Stages<16>::bytes + 256;
      cudaFuncSetAttribute(k_coarse_apply_tc4<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      k_coarse_apply_tc4<16><<<grid, TC_THREADS + 32, smem, st>>>(out, *Bt, *At4, Lc[0], Lc[1], Lc[2], Lc[3],
                                                                   nquads, err_dev);
    } else {
      smem = Tc4Stages<32>::v * Tc4Stages<32>::bytes + 256;
      cudaFuncSetAttribute(k_coarse_apply_tc4<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      k_coarse_apply_tc4<32><<<grid, TC_THREADS + 32, smem, st>>>(out, *Bt, *At4, Lc[0], Lc[1], Lc[2], Lc[3],
                                                                   nquads, err_dev);
    }
    return DWF_OK;
  }
  if (!*At) {
    if (cudaMalloc(At, (size_t)nc * 9 * TC_ROWS * TC_ROWS * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return DWF_ENOMEM;
    }
    const long long n = (long long)nc * 9 * TC_ROWS * TC_ROWS;
    k_tc_arrange<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(*At, A32, nc);
    c->launches++;
  }
  const size_t bbytes = (size_t)nc * TC_ROWS * nrhs * sizeof(float);
  if (*Bt_bytes < bbytes) {
    if (*Bt) cudaFree(*Bt);
    *Bt = nullptr;
    *Bt_bytes = 0;
    if (cudaMalloc(Bt, bbytes) != cudaSuccess) {
      cudaGetLastError();
      return DWF_ENOMEM;
    }
    *Bt_bytes = bbytes;
  }
  {
    const long long n = (long long)nc * TC_NB * nrhs;
    k_tc_arrange_in<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(*Bt, in, nc, nrhs);
    c->launches++;
  }
  const int npairs = nc / 2;
  const int grid = npairs < nsm ? npairs : nsm;
  c->launches++;
#define DWF_TC_CASE(NV)                                                                                      \
  case NV:                                                                                                   \
    smem = TcStages<NV>::v * TcStages<NV>::bytes + 256;                                                      \
    cudaFuncSetAttribute(k_coarse_apply_tc<NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);          \
    k_coarse_apply_tc<NV><<<grid, TC_THREADS + 32, smem, st>>>(out, *Bt, *At, Lc[0], Lc[1], Lc[2], Lc[3],    \
                                                               npairs, err_dev);                             \
    break;
  int smem = 0;
  switch (nrhs) {
    DWF_TC_CASE(16)
    DWF_TC_CASE(32)
    DWF_TC_CASE(64)
  }
#undef DWF_TC_CASE
  return DWF_OK;
}
