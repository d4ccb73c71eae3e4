// peak.cu -- measured arithmetic peaks for the roofline of the step kernels.
//
// The FP64 path of the step is bound by FP64 arithmetic on this part, not by memory, so its
// roofline needs the device's FP64 fused-multiply-add rate.  fma_rate_kernel runs kChains
// independent FMA chains per thread (enough instruction-level parallelism to keep the FMA pipes
// busy) for a fixed number of iterations; the rate is 2 flops per FMA over the elapsed time of
// the launch, measured with CUDA events on the caller's stream.  Nothing is waited on inside the
// kernel; the loop bounds are compile-time constants.
#include <cuda_runtime.h>

#include "../../include/fdtdbath.h"

namespace {

constexpr int kChains = 16;
constexpr int kIters = 2048;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_rate_kernel(T seed, T* out) {
  T acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = seed + T(c) * T(1e-3) + T(threadIdx.x) * T(1e-6);
  const T a = T(0.999999), b = T(1e-7);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == T(-1)) out[blockIdx.x] = s;   // keeps the chains live; never true for these inputs
}

template <typename T>
int measure(int device, int reps, double* flops_per_s) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return FDTDBATH_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
    return FDTDBATH_ERR_CUDA;
  const int blocks = sms * 8;   // 2048 threads per SM
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks) != cudaSuccess) return FDTDBATH_ERR_OOM;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 0.0f;
  for (int r = 0; r < reps + 1; ++r) {   // the first launch warms up
    cudaEventRecord(a);
    fma_rate_kernel<T><<<blocks, kThreads>>>(T(0.5), out);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    if (r > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess || best <= 0.0f) return FDTDBATH_ERR_CUDA;
  const double fmas = (double)blocks * kThreads * kChains * kIters;
  *flops_per_s = 2.0 * fmas / (best * 1e-3);
  return FDTDBATH_OK;
}

}  // namespace

extern "C" int fdtdbath_measure_fma_rate(int32_t precision, int32_t device, int32_t reps, double* flops_per_s) {
  if (!flops_per_s || reps < 1 || (precision != 32 && precision != 64)) return FDTDBATH_ERR_ARG;
  return precision == 64 ? measure<double>(device, reps, flops_per_s) : measure<float>(device, reps, flops_per_s);
}
