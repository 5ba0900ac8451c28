// Allocation-free convolve-and-subtract: sfft_apply_noalloc.
//
// Who needs it: callers that must not allocate device memory themselves, for
// example code that runs where the allocator is off limits (inside another
// library's memory-managed region, in a real-time loop with a fixed memory
// budget, or in a process whose allocations are owned by a framework it
// cannot call into).  They cannot create a plan (sfft_plan allocates its
// tables) or hand over a workspace, so this entry point takes explicit shapes
// and needs only the caller's inputs and output.
//
// Its one piece of scratch is the theta vector converted to offset units
// (N doubles per CCD).  That scratch lives in the file-scope device array
// below, of fixed size: every GPU that loads this library holds it until the
// process exits, and every call shares it.
#include <mutex>

#include "common.cuh"
#include "plan.h"

namespace {

// batch * N must not exceed this many doubles (64 CCDs at the largest model,
// N = 11*11*6 + 6 = 732), i.e. 375 KB per device.
constexpr int64_t kNoallocMaxTheta = 64 * 732;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_theta_off[kNoallocMaxTheta];

std::mutex g_setup_mu;
double* g_scratch[kMaxDevices] = {};

// Device address of the scratch array for the current device.  The host
// symbol is only a stand-in: kernels must be given this address instead.
sfft_status_t scratch_for_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    sfft::set_last_error(cudaGetErrorString(e));
    return SFFT_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    sfft::set_last_error("sfft_apply_noalloc: device index beyond the supported range");
    return SFFT_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_theta_off);
    if (e != cudaSuccess || p == nullptr) {
      sfft::set_last_error(e != cudaSuccess ? cudaGetErrorString(e) : "cudaGetSymbolAddress returned null");
      return SFFT_ERR_CUDA;
    }
    g_scratch[dev] = static_cast<double*>(p);
  }
  *out = g_scratch[dev];
  return SFFT_OK;
}

}  // namespace

extern "C" sfft_status_t sfft_apply_noalloc(int32_t H, int32_t W, int32_t L, int32_t DK, int32_t DB, int32_t batch,
                                            int32_t prec, const float* R, const float* S, const double* theta,
                                            const double* sky, float* D, void* cuda_stream) {
  if (!R || !S || !theta || !sky || !D) {
    sfft::set_last_error("sfft_apply_noalloc: R, S, theta, sky and D are required");
    return SFFT_ERR_ARG;
  }
  if (H <= 0 || W <= 0 || batch <= 0 || L <= 0 || (prec != SFFT_PREC_FP64 && prec != SFFT_PREC_MIXED)) {
    sfft::set_last_error("sfft_apply_noalloc: invalid shape or precision");
    return SFFT_ERR_ARG;
  }
  if ((L & 1) == 0 || L > sfft::kMaxL || DK < 0 || DB < 0 || DK > sfft::kMaxD || DB > sfft::kMaxD || H < L ||
      W < L) {
    sfft::set_last_error("sfft_apply_noalloc: L must be odd and <= 11, 0 <= D_K, D_B <= 2, H and W >= L");
    return SFFT_ERR_UNSUPPORTED;
  }
  const int NK = sfft::n_mono(DK), NB = sfft::n_mono(DB);
  const int64_t N = (int64_t)L * L * NK + NB;
  if (N * batch > kNoallocMaxTheta) {
    sfft::set_last_error("sfft_apply_noalloc: batch * N exceeds the fixed scratch of 46848 doubles "
                         "(e.g. at most 64 CCDs at L = 11, D_K = D_B = 2)");
    return SFFT_ERR_UNSUPPORTED;
  }
  double* scratch = nullptr;
  sfft_status_t st = scratch_for_current_device(&scratch);
  if (st != SFFT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // theta (background in original units) -> offset units; fully overwrites the
  // scratch rows it uses, so nothing needs clearing between calls
  cudaError_t e = sfft::launch_theta_units_raw(s, theta, scratch, sky, L, NK, NB, batch, 0);
  if (e == cudaSuccess)
    e = sfft::launch_apply_raw(s, prec == SFFT_PREC_FP64, R, S, scratch, sky, D, H, W, L, DK, DB, batch);
  if (e != cudaSuccess) {
    sfft::set_last_error(cudaGetErrorString(e));
    return SFFT_ERR_CUDA;
  }
  return SFFT_OK;
}
