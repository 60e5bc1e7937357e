// Coarse 9-point stencil on the 5th-generation tensor cores (tcgen05, TF32
// inputs, FP32 accumulation in tensor memory): out(x) = sum_d A_d(x) in(x+d)
// for many right-hand sides (Sec. 3.1, Eq. 18: the little Dirac operator is a
// dense nb x nb block stencil, a real dense contraction).
//
// Real form of one complex block product (nb = 32):
//   [Re out; Im out] (64 x N) = [[Ar, -Ai], [Ai, Ar]] (64 x 64) [Re in; Im in] (64 x N)
// tcgen05.mma with M = 128 is used with two coarse sites per CTA packed
// block-diagonally: rows 0-63 / K 0-63 belong to site x1, rows 64-127 /
// K 64-127 to site x2 (the off-diagonal blocks are zero and stay resident in
// shared memory), so the accumulator row i is TMEM lane i.  For each of the 9
// directions one pipeline stage holds
//   A: [K/4 = 32][M = 128][4] TF32 (64 KB; the two 16 KB site blocks arrive by
//      cp.async.bulk from a pre-arranged copy of the operator)
//   B: [K/4 = 32][N][4] TF32 (N*512 B; the neighbours' input vectors, split
//      into real and imaginary rows by the threads)
// in the canonical no-swizzle K-major layout (8-row x 16-byte core matrices;
// K-adjacent cores LBO apart, M/N-adjacent cores 128 B apart).  16 MMAs of
// K = 8 per stage, two stages in flight, one tcgen05.commit per stage.
#include <string.h>

#include "dwf_internal.cuh"
#include "mg_kernels.cuh"

namespace {

constexpr int TC_NB = 32;           // basis vectors per site handled here
constexpr int TC_ROWS = 2 * TC_NB;  // real rows per site
constexpr int TC_M = 128;
constexpr int TC_K = 128;           // per stage: two sites x 64
constexpr int TC_THREADS = 128;
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

// Pre-arranged operator: At[x][d][kg = 16][r = 64][4] TF32 (real form, K-major).
__global__ void k_tc_arrange(float* At, const float2* A, int nc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // (x, d, r, k)
  if (e >= (long long)nc * 9 * TC_ROWS * TC_ROWS) return;
  const int k = (int)(e % TC_ROWS);
  const int r = (int)((e / TC_ROWS) % TC_ROWS);
  const long long xd = e / (TC_ROWS * TC_ROWS);
  const int j = r % TC_NB, kk = k % TC_NB;
  const float2 a = A[(xd * TC_NB + j) * TC_NB + kk];
  float v;
  if (r < TC_NB)
    v = k < TC_NB ? a.x : -a.y;
  else
    v = k < TC_NB ? a.y : a.x;
  At[((xd * (TC_ROWS / 4) + k / 4) * TC_ROWS + r) * 4 + (k & 3)] = to_tf32(v);
}

template <int N>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_coarse_apply_tc(float2* out, const float2* in, const float* At, int Lc0, int Lc1, int Lc2, int Lc3,
                      int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int A_BYTES = (TC_K / 4) * TC_M * 16;  // 64 KB
  constexpr int B_BYTES = (TC_K / 4) * N * 16;
  constexpr uint32_t LBO_A = TC_M * 16, LBO_B = N * 16, SBO = 128;
  unsigned char* Abuf[2] = {smem, smem + A_BYTES};
  unsigned char* Bbuf[2] = {smem + 2 * A_BYTES, smem + 2 * A_BYTES + B_BYTES};
  uint64_t* bars = (uint64_t*)(smem + 2 * A_BYTES + 2 * B_BYTES);  // full[2], done[2]
  uint32_t* tslot = (uint32_t*)(bars + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Lc[4] = {Lc0, Lc1, Lc2, Lc3};
  const int nc = Lc0 * Lc1 * Lc2 * Lc3;
  const int x1 = 2 * blockIdx.x, x2 = 2 * blockIdx.x + 1;
  const int xs[2] = {x1, x2};

  // zero both A stages (the off-diagonal blocks stay zero)
  for (int i = tid; i < 2 * A_BYTES / 16; i += TC_THREADS) ((uint4*)smem)[i] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int i = 0; i < 4; i++) mbar_init(smem_u32(bars + i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(32 * ((N + 31) / 32)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
                             ((uint32_t)(TC_M >> 4) << 24);
  bool ok = true;

  for (int d = 0; d < 9; d++) {
    const int buf = d & 1;
    const uint32_t use = (uint32_t)(d >> 1) & 1u;
    if (d >= 2) {  // the MMAs of stage d-2 have finished reading this buffer
      if (!mbar_wait(smem_u32(bars + 2 + buf), use ^ 1u)) ok = false;
    }
    __syncthreads();
    if (ok && tid == 0) {
      const uint32_t fb = smem_u32(bars + buf);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(2 * 16 * 1024) : "memory");
      for (int q = 0; q < 2; q++) {
        const float* src = At + ((long long)xs[q] * 9 + d) * (TC_ROWS / 4) * TC_ROWS * 4;
        for (int kg = 0; kg < 16; kg++) {
          const uint32_t dst = smem_u32(Abuf[buf] + (size_t)(16 * q + kg) * LBO_A + q * TC_ROWS * 16);
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
              "l"(src + kg * TC_ROWS * 4), "r"(TC_ROWS * 16), "r"(fb)
              : "memory");
        }
      }
    }
    // B: neighbours' inputs, split into real (k = j) and imaginary (k = 32 + j) rows
    float* B = (float*)Bbuf[buf];
    for (int e = tid; e < 2 * TC_NB * N; e += TC_THREADS) {
      const int n = e % N, j = (e / N) % TC_NB, q = e / (N * TC_NB);
      const int y = dwfmg::coarse_nbr(Lc, xs[q], d);
      const float2 v = in[((long long)y * TC_NB + j) * N + n];
      const int kre = 64 * q + j, kim = 64 * q + 32 + j;
      B[((kre >> 2) * N + n) * 4 + (kre & 3)] = to_tf32(v.x);
      B[((kim >> 2) * N + n) * 4 + (kim & 3)] = to_tf32(v.y);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (ok && tid == 0) {
      if (!mbar_wait(smem_u32(bars + buf), use)) {
        ok = false;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(Abuf[buf]), b0 = smem_u32(Bbuf[buf]);
#pragma unroll
        for (int kk = 0; kk < TC_K / 8; kk++) {
          const uint64_t ad = smem_desc(a0 + kk * 2 * LBO_A, LBO_A, SBO);
          const uint64_t bd = smem_desc(b0 + kk * 2 * LBO_B, LBO_B, SBO);
          const uint32_t acc = (d > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(bars + 2 + buf))
                     : "memory");
      }
    }
    if (tid == 0 && !ok) atomicExch(err, 1);
    ok = __syncthreads_and(ok);
  }
  // the last commit (stage 8, buffer 0, fifth use) covers every earlier MMA
  if (ok && !mbar_wait(smem_u32(bars + 2), 0u)) ok = false;
  if (!ok && tid == 0) {
    atomicExch(err, 1);
    mbar_wait(smem_u32(bars + 0), 0u);  // bounded: let copies in flight land
    mbar_wait(smem_u32(bars + 1), 1u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // each warp reads its 32 TMEM lanes (= accumulator rows) across N columns
    const int r = warp * 32 + lane;
    const int q = r / TC_ROWS, rr = r % TC_ROWS;
    const int part = rr / TC_NB, j = rr % TC_NB;
    float* o = (float*)(out + ((long long)xs[q] * TC_NB + j) * N) + part;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 16; i++) o[2 * (c0 + i)] = __uint_as_float(v[i]);
    }
  }
  (void)nc;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32 * ((N + 31) / 32)));
  }
}

}  // namespace

// Tensor-core coarse apply; returns DWF_EINVAL when the shape is not covered
// (nb != 32, an odd number of coarse sites, nrhs not 16, 32 or 64).
int coarse_apply_tc(dwf_ctx* c, float2* out, const float2* in, const float2* A32, float** At, int nb, int nc,
                    const int Lc[4], int nrhs, int* err_dev, cudaStream_t st) {
  if (nb != TC_NB || (nc & 1) || (nrhs != 16 && nrhs != 32 && nrhs != 64)) return DWF_EINVAL;
  if (!*At) {
    if (cudaMalloc(At, (size_t)nc * 9 * TC_ROWS * TC_ROWS * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return DWF_ENOMEM;
    }
    const long long n = (long long)nc * 9 * TC_ROWS * TC_ROWS;
    k_tc_arrange<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(*At, A32, nc);
    c->launches++;
  }
  const int smem = 2 * (TC_K / 4) * TC_M * 16 + 2 * (TC_K / 4) * nrhs * 16 + 64;
  c->launches++;
  switch (nrhs) {
    case 16:
      cudaFuncSetAttribute(k_coarse_apply_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      k_coarse_apply_tc<16><<<nc / 2, TC_THREADS, smem, st>>>(out, in, *At, Lc[0], Lc[1], Lc[2], Lc[3], err_dev);
      break;
    case 32:
      cudaFuncSetAttribute(k_coarse_apply_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      k_coarse_apply_tc<32><<<nc / 2, TC_THREADS, smem, st>>>(out, in, *At, Lc[0], Lc[1], Lc[2], Lc[3], err_dev);
      break;
    default:
      cudaFuncSetAttribute(k_coarse_apply_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      k_coarse_apply_tc<64><<<nc / 2, TC_THREADS, smem, st>>>(out, in, *At, Lc[0], Lc[1], Lc[2], Lc[3], err_dev);
      break;
  }
  return DWF_OK;
}
