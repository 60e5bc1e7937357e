// Measured FMA rates of this GPU's CUDA cores in FP64 and FP32, the ALU roof
// against which the FP64 hopping kernel (and the FP64 parts of the solvers)
// are reported.  The paper has no counterpart: it is the measurement that
// replaces a spec-sheet figure.
//
// Each thread runs 8 independent fused multiply-add chains for `iters`
// steps (a -> a * m + k with |m| < 1, so the values stay finite and do not
// denormalise), on a grid of 8 CTAs of 256 threads per SM; every FMA counts
// 2 flops.  The chains' final values are summed into a device word so that
// the compiler cannot drop them.
#include <cuda_runtime.h>

#include "dwf_internal.cuh"

namespace {

constexpr int AP_THREADS = 256;
constexpr int AP_CHAINS = 8;

template <class T>
__global__ void __launch_bounds__(AP_THREADS) k_fma_chains(int iters, T m, T k, T* sink) {
  T a[AP_CHAINS];
#pragma unroll
  for (int j = 0; j < AP_CHAINS; j++) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int j = 0; j < AP_CHAINS; j++) a[j] = fma(a[j], m, k);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < AP_CHAINS; j++) s += a[j];
  if (s == (T)-1) *sink = s;  // never true; keeps the chains live
}

template <class T>
int time_chains(int grid, int iters, double* tflops, cudaStream_t st) {
  T* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return DWF_ENOMEM;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(sink);
    return DWF_ECUDA;
  }
  const T m = (T)0.999999, k = (T)1e-6;
  k_fma_chains<T><<<grid, AP_THREADS, 0, st>>>(iters / 8, m, k, sink);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 3; r++) {
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<grid, AP_THREADS, 0, st>>>(iters, m, k, sink);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return DWF_ECUDA;
  const double flops = 2.0 * AP_CHAINS * (double)iters * AP_THREADS * grid;
  *tflops = flops / (best * 1e-3) / 1e12;
  return DWF_OK;
}

}  // namespace

extern "C" int dwf_measure_fma_peaks(double* fp64_tflops, double* fp32_tflops, void* stream) {
  if (!fp64_tflops || !fp32_tflops) return DWF_EINVAL;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return DWF_ECUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = nsm * 8;
  int rc = time_chains<double>(grid, 1 << 14, fp64_tflops, st);
  if (rc) return rc;
  return time_chains<float>(grid, 1 << 16, fp32_tflops, st);
}
