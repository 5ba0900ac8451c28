// Measured arithmetic peaks for the roofline reports: the FP32 and FP64
// FMA rates of this GPU, from a kernel of independent FMA chains.
//
// Each thread keeps kChains independent accumulators and applies
// a <- a * b + c to each of them kIters times (b, c loop invariant), so the
// FMA pipes see kChains independent instructions back to back; the grid puts
// 8 CTAs of 256 threads on every SM.  The rate is 2 x FMAs / time (CUDA
// events around one launch after a warm-up launch).  The results are stored,
// so the chains are not optimised away.
#include "common.cuh"
#include "plan.h"

namespace sfft {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* out, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i) * (T)1e-3;
#pragma unroll 1
  for (int it = 0; it < kIters; it += 16) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = (T)0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
sfft_status_t measure(cudaStream_t s, double* tflops) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms * 8;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)grid * kThreads) != cudaSuccess) {
    cudaGetLastError();
    return SFFT_ERR_NOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sfft_status_t st = SFFT_ERR_CUDA;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
    // b slightly below one keeps the chains bounded
    k_fma_chains<T><<<grid, kThreads, 0, s>>>(out, (T)0.999, (T)1e-3);
    cudaEventRecord(e0, s);
    k_fma_chains<T><<<grid, kThreads, 0, s>>>(out, (T)0.999, (T)1e-3);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f) {
      const double fmas = (double)grid * kThreads * kChains * kIters;
      *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
      st = SFFT_OK;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (st != SFFT_OK) cudaGetLastError();
  return st;
}

}  // namespace
}  // namespace sfft

extern "C" sfft_status_t sfft_probe_fma_peak(int32_t fp64, double* tflops, void* cuda_stream) {
  if (!tflops) return SFFT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return fp64 ? sfft::measure<double>(s, tflops) : sfft::measure<float>(s, tflops);
}
