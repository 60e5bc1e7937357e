// Self-test of the bounded device waits (failure detection without a GPU
// fault): the two wait forms the library's kernels use -- polling a global
// counter (the grid barrier of the persistent coarse CG) and an mbarrier
// phase (the tensor-core pipeline) -- are made to wait on something that never
// arrives, with a short limit, and must give up, report and return.
#include <cuda_runtime.h>

#include "dwf_internal.cuh"

namespace {

// Polls *flag (never set) at most `limit` times with a short pause; records
// in out[0] whether it gave up.
__global__ void k_poll_timeout(const unsigned* flag, unsigned limit, int* out) {
  if (threadIdx.x != 0) return;
  int arrived = 0;
  for (unsigned i = 0; i < limit; i++) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v != 0u) {
      arrived = 1;
      break;
    }
    __nanosleep(64);
  }
  out[0] = arrived ? 0 : 1;
}

// Waits at most `limit` tries for phase 0 of an mbarrier that expects one
// arrival nobody makes; records in out[1] whether it gave up.
__global__ void k_mbar_timeout(unsigned limit, int* out) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned b = (unsigned)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(1u));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  int done = 0;
  for (unsigned i = 0; i < limit && !done; i++) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(b), "r"(0u)
        : "memory");
    done = (int)ok;
  }
  out[1] = done ? 0 : 1;
}

}  // namespace

extern "C" int dwf_selftest_wait_timeout(int* gave_up, void* stream) {
  if (!gave_up) return DWF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* flag = nullptr;
  int* out = nullptr;
  if (cudaMalloc(&flag, sizeof(unsigned)) != cudaSuccess || cudaMalloc(&out, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (flag) cudaFree(flag);
    return DWF_ENOMEM;
  }
  int rc = DWF_OK;
  if (cudaMemsetAsync(flag, 0, sizeof(unsigned), st) != cudaSuccess ||
      cudaMemsetAsync(out, 0xff, 2 * sizeof(int), st) != cudaSuccess)
    rc = DWF_ECUDA;
  if (!rc) {
    k_poll_timeout<<<1, 32, 0, st>>>(flag, 1u << 14, out);  // about 1 ms of polling
    k_mbar_timeout<<<1, 32, 0, st>>>(1u << 14, out);
    int h[2] = {-1, -1};
    if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = DWF_ECUDA;
    } else {
      gave_up[0] = h[0];
      gave_up[1] = h[1];
      rc = (h[0] == 1 && h[1] == 1) ? DWF_ETIMEOUT : DWF_OK;
    }
  }
  cudaFree(flag);
  cudaFree(out);
  return rc;
}
