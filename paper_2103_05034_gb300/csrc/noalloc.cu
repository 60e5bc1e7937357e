// Allocation-free norm^2 for callers that cannot call cudaMalloc.
//
// Some callers cannot allocate device memory at the point where they need a
// global reduction: code running inside a memory pool that forbids
// cudaMalloc/cudaFree, library plug-ins handed only input and output
// buffers, or code paths that must not trigger the implicit device
// synchronisation an allocation can cause.  dwf_norm2_noalloc serves them: it
// keeps its reduction scratch (one FP64 partial sum per CTA, plus the final
// sum) in a file-scope __device__ array that is part of the loaded library
// image, so the call itself allocates nothing.  The array costs 512 KiB + 8 B
// on every GPU that loads the library, until the process exits.
//
// Limits and sharing:
//  * n (complex numbers) may be at most DWF_NOALLOC_MAX_N = 2^31: each CTA
//    reduces a fixed chunk of 32768 complex numbers and the scratch holds
//    65536 partial sums; larger n is rejected with DWF_EINVAL.
//  * every call on a device uses the same scratch: two calls that overlap on
//    the GPU (different streams, or concurrent host threads) race and may
//    return wrong sums.  Serialise them (one stream, or events).
//  * the first call on a device looks up the device address of the scratch
//    (cudaGetSymbolAddress, with that device current) and caches it; make that
//    first call before any stream capture.  The cached address belongs to the
//    device's primary context: after cudaDeviceReset (or any other teardown of
//    that context) in the same process, this entry point must not be used
//    again on that device.
#include <mutex>

#include "dwf_internal.cuh"

#define DWF_NOALLOC_CHUNK 32768LL
#define DWF_NOALLOC_MAXPART 65536
#define DWF_NOALLOC_MAX_N (DWF_NOALLOC_CHUNK * DWF_NOALLOC_MAXPART)
#define DWF_NOALLOC_MAXDEV 64

// [0, MAXPART): per-CTA partial sums; [MAXPART]: the final sum.
static __device__ __align__(256) double g_noalloc_scratch[DWF_NOALLOC_MAXPART + 1];

namespace {

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[DWF_NOALLOC_MAXDEV] = {nullptr};

constexpr int NT = 256;

__device__ __forceinline__ double warp_block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; i++) t += sh[i];
  return t;
}

// CTA b sums |a|^2 over complex numbers [b*CHUNK, min(n, (b+1)*CHUNK)).
template <int P>
__global__ void __launch_bounds__(NT) k_noalloc_partial(const typename Prec<P>::S* a, long long n, double* scratch) {
  __shared__ double sh[NT / 32];
  const long long lo = (long long)blockIdx.x * DWF_NOALLOC_CHUNK;
  const long long hi = lo + DWF_NOALLOC_CHUNK < n ? lo + DWF_NOALLOC_CHUNK : n;
  double acc = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += NT) {
    const auto z = ld_c(a + i);
    acc += (double)z.re * z.re + (double)z.im * z.im;
  }
  const double t = warp_block_sum(acc, sh);
  if (threadIdx.x == 0) scratch[blockIdx.x] = t;
}

// One CTA adds the nparts partial sums in a fixed order into scratch[MAXPART].
__global__ void __launch_bounds__(NT) k_noalloc_final(int nparts, double* scratch) {
  __shared__ double sh[NT / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += NT) acc += scratch[i];
  const double t = warp_block_sum(acc, sh);
  if (threadIdx.x == 0) scratch[DWF_NOALLOC_MAXPART] = t;
}

// Device address of the scratch on the current device (looked up once).
int noalloc_scratch(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DWF_ECUDA;
  if (dev < 0 || dev >= DWF_NOALLOC_MAXDEV) return DWF_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return DWF_ECUDA;
    }
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return DWF_OK;
}

}  // namespace

extern "C" int dwf_norm2_noalloc(double* result, const void* a, int64_t n, int prec, void* stream) {
  if (!result || (!a && n > 0) || n < 0) return DWF_EINVAL;
  if (n > DWF_NOALLOC_MAX_N) return DWF_EINVAL;  // beyond the scratch capacity
  if (prec != DWF_F64 && prec != DWF_F32 && prec != DWF_F16S) return DWF_EINVAL;
  if (n == 0) {
    *result = 0.0;
    return DWF_OK;
  }
  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nparts = (int)((n + DWF_NOALLOC_CHUNK - 1) / DWF_NOALLOC_CHUNK);
  switch (prec) {
    case DWF_F64:
      k_noalloc_partial<DWF_F64><<<nparts, NT, 0, st>>>((const double2*)a, n, scratch);
      break;
    case DWF_F32:
      k_noalloc_partial<DWF_F32><<<nparts, NT, 0, st>>>((const float2*)a, n, scratch);
      break;
    default:
      k_noalloc_partial<DWF_F16S><<<nparts, NT, 0, st>>>((const __half2*)a, n, scratch);
      break;
  }
  // a launch that failed (no kernel image, bad stream) would leave the last
  // call's sum in the scratch: report it instead of returning a stale result
  if (cudaGetLastError() != cudaSuccess) return DWF_ECUDA;
  k_noalloc_final<<<1, NT, 0, st>>>(nparts, scratch);
  if (cudaGetLastError() != cudaSuccess) return DWF_ECUDA;
  if (cudaMemcpyAsync(result, scratch + DWF_NOALLOC_MAXPART, sizeof(double), cudaMemcpyDeviceToHost, st) !=
      cudaSuccess) {
    cudaGetLastError();
    return DWF_ECUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return DWF_ECUDA;
  }
  return DWF_OK;
}
