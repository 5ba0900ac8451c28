// Measured arithmetic peaks for the roofline reports: the FP32 and FP64
// FMA rates of this GPU, from a kernel of independent FMA chains; and the
// cycles one tcgen05 MMA with both operands in shared memory takes, by N.
//
// Each thread keeps kChains independent accumulators and applies
// a <- a * b + c to each of them kIters times (b, c loop invariant), so the
// FMA pipes see kChains independent instructions back to back; the grid puts
// 8 CTAs of 256 threads on every SM.  The rate is 2 x FMAs / time (CUDA
// events around one launch after a warm-up launch).  The results are stored,
// so the chains are not optimised away.
#include "common.cuh"
#include "plan.h"
#include "umma_common.cuh"

#include <vector>

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

// Back-to-back tcgen05.mma (kind::f16, BF16, M = 128, K = 16, FP32
// accumulation in tensor memory, A and B from shared memory in the canonical
// K-major layout without swizzle) issued by one thread per CTA, one CTA per
// SM: the issuing thread's clock from the first issue to the completion of
// the last (tracked by an mbarrier; the wait is bounded and a wait that gives
// up reports -1).  The operands hold BF16 ones (sums stay finite).
constexpr int kUmmaIters = 2000;
constexpr int kUmmaSmem = 96 * 1024;   // A at 0 (<= 8 KB read), B at 64 KB (<= 8 KB)

__global__ void __launch_bounds__(128) k_umma_rate(int n, long long* out) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tb;
  for (int i = threadIdx.x; i < kUmmaSmem / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(sm)[i] = 0x3f803f80u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tb)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t t = tb;
  if (threadIdx.x == 0) {
    const uint64_t ad = smem_desc_kn(smem_u32(sm), 2048, 128);
    const uint64_t bd = smem_desc_kn(smem_u32(sm) + 64 * 1024, 16 * n, 128);
    const uint32_t id = instr_desc(1, (uint32_t)n);
    const long long t0 = clock64();
    for (int i = 0; i < kUmmaIters; ++i)
      asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                   " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                   ::"r"(t), "l"(ad), "l"(bd), "r"(id), "r"(i > 0 ? 1u : 0u) : "memory");
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar))
                 : "memory");
    const bool ok = mbar_wait_bounded(&bar, 0);
    out[blockIdx.x] = ok ? clock64() - t0 : -1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(t) : "memory");
}

sfft_status_t measure_umma(int n, cudaStream_t s, double* cycles) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaFuncSetAttribute(k_umma_rate, cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaSmem) != cudaSuccess)
    return SFFT_ERR_CUDA;
  long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(long long) * sms) != cudaSuccess) {
    cudaGetLastError();
    return SFFT_ERR_NOMEM;
  }
  std::vector<long long> h(sms);
  k_umma_rate<<<sms, 128, kUmmaSmem, s>>>(n, d);   // warm-up
  k_umma_rate<<<sms, 128, kUmmaSmem, s>>>(n, d);
  sfft_status_t st = SFFT_ERR_CUDA;
  if (cudaStreamSynchronize(s) == cudaSuccess &&
      cudaMemcpy(h.data(), d, sizeof(long long) * sms, cudaMemcpyDeviceToHost) == cudaSuccess) {
    double sum = 0.0;
    st = SFFT_OK;
    for (long long v : h) {
      if (v < 0) st = SFFT_ERR_TIMEOUT;
      sum += (double)v;
    }
    if (st == SFFT_OK) *cycles = sum / sms / kUmmaIters;
  }
  cudaFree(d);
  if (st == SFFT_ERR_CUDA) cudaGetLastError();
  return st;
}

}  // namespace
}  // namespace sfft

extern "C" sfft_status_t sfft_probe_umma_cycles(int32_t n, double* cycles_per_mma, void* cuda_stream) {
  if (!cycles_per_mma || n < 16 || n > 256 || n % 16) return SFFT_ERR_ARG;
  return sfft::measure_umma(n, static_cast<cudaStream_t>(cuda_stream), cycles_per_mma);
}

extern "C" sfft_status_t sfft_probe_fma_peak(int32_t fp64, double* tflops, void* cuda_stream) {
  if (!tflops) return SFFT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  return fp64 ? sfft::measure<double>(s, tflops) : sfft::measure<float>(s, tflops);
}
