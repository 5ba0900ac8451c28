// Differential photometry on difference images: forced aperture fluxes, the
// limiting-magnitude Monte Carlo and the multi-template median combination.
// One warp per aperture: lanes walk the aperture's bounding box, each pixel's
// weight counts the 5 x 5 sub-pixel centres inside the disc with IEEE double
// operations that are never fused (so the inside/outside decisions are those
// of any other IEEE evaluation of the same expression), and the weighted sum
// is reduced in FP64 across the warp.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "phot.h"
#include "plan.h"

namespace {

constexpr int kSub = 5;

__device__ __forceinline__ double sub_offset(int j) { return __ddiv_rn((double)j + 0.5, (double)kSub); }

__global__ void __launch_bounds__(256)
k_aperture(int H, int W, int batch, const float* __restrict__ D, const uint8_t* __restrict__ bad,
           const double* __restrict__ pos, int n, double r, double* __restrict__ flux, int32_t* __restrict__ flag) {
  const int lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= (int64_t)batch * n) return;   // whole warps
  const int c = (int)(item / n);
  const double xc = pos[2 * item], yc = pos[2 * item + 1];
  const double r2 = __dmul_rn(r, r);
  const int x0 = (int)floor(__dadd_rn(__dadd_rn(xc, -r), -1.0)), x1 = (int)ceil(__dadd_rn(__dadd_rn(xc, r), 1.0));
  const int y0 = (int)floor(__dadd_rn(__dadd_rn(yc, -r), -1.0)), y1 = (int)ceil(__dadd_rn(__dadd_rn(yc, r), 1.0));
  const int nx = x1 - x0 + 1, ny = y1 - y0 + 1;
  const int64_t img = (int64_t)H * W;
  const float* Dc = D + c * img;
  const uint8_t* bc = bad ? bad + c * img : nullptr;
  double s = 0.0;
  int fl = 0;
  for (int p = lane; p < nx * ny; p += 32) {
    const int yy = y0 + p / nx, xx = x0 + p % nx;
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < kSub; ++j) {
      const double dy = __dadd_rn(__dadd_rn((double)yy - 0.5, sub_offset(j)), -yc);
      const double dy2 = __dmul_rn(dy, dy);
#pragma unroll
      for (int i = 0; i < kSub; ++i) {
        const double dx = __dadd_rn(__dadd_rn((double)xx - 0.5, sub_offset(i)), -xc);
        cnt += __dadd_rn(dy2, __dmul_rn(dx, dx)) <= r2 ? 1 : 0;
      }
    }
    if (cnt == 0) continue;
    if (yy < 0 || yy >= H || xx < 0 || xx >= W) {
      fl = 1;
      continue;
    }
    const int64_t q = (int64_t)yy * W + xx;
    const float v = Dc[q];
    if (!isfinite(v) || (bc && bc[q])) {
      fl = 1;
      continue;
    }
    s += __ddiv_rn((double)cnt, (double)(kSub * kSub)) * (double)v;
  }
  s = sfft::warp_sum(s);
  fl = __reduce_or_sync(0xffffffffu, (unsigned)fl);
  if (lane == 0) {
    flux[item] = s;
    flag[item] = fl;
  }
}

// per CCD: mean and sample standard deviation of the unflagged fluxes (two
// passes, fixed-order reductions), then the 5-sigma limiting magnitude
__global__ void __launch_bounds__(256)
k_limit(const double* __restrict__ flux, const int32_t* __restrict__ flag, int n, double zp,
        double* __restrict__ sigma, double* __restrict__ mlim, int32_t* __restrict__ ngood) {
  __shared__ double red[256];
  __shared__ int redn[256];
  const int c = blockIdx.x, t = threadIdx.x;
  const double* f = flux + (int64_t)c * n;
  const int32_t* g = flag + (int64_t)c * n;
  double s = 0.0;
  int m = 0;
  for (int i = t; i < n; i += blockDim.x)
    if (!g[i]) { s += f[i]; ++m; }
  red[t] = s;
  redn[t] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) { red[t] += red[t + o]; redn[t] += redn[t + o]; }
    __syncthreads();
  }
  const int cnt = redn[0];
  const double mean = red[0] / (double)cnt;
  __syncthreads();
  double q = 0.0;
  for (int i = t; i < n; i += blockDim.x)
    if (!g[i]) { const double d = f[i] - mean; q += d * d; }
  red[t] = q;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (t < o) red[t] += red[t + o];
    __syncthreads();
  }
  if (t == 0) {
    const double sd = cnt > 1 ? sqrt(red[0] / (double)(cnt - 1)) : (double)NAN;
    sigma[c] = sd;
    mlim[c] = sd > 0.0 ? zp - 2.5 * log10(5.0 * sd) : (double)NAN;
    ngood[c] = cnt;
  }
}

constexpr int kMaxTemplates = 16;

__global__ void __launch_bounds__(256)
k_median_combine(int64_t npx, int ntemp, const float* __restrict__ D, const float* __restrict__ scale,
                 const uint8_t* __restrict__ bad, float* __restrict__ out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npx; p += (int64_t)gridDim.x * blockDim.x) {
    float v[kMaxTemplates];
    int cnt = 0;
    for (int t = 0; t < ntemp; ++t) {
      const float d = D[t * npx + p];
      if (!isfinite(d) || (bad && bad[t * npx + p])) continue;
      float x = scale[t] * d;
      int j = cnt++;
      for (; j > 0 && v[j - 1] > x; --j) v[j] = v[j - 1];   // insertion sort
      v[j] = x;
    }
    float m = NAN;
    if (cnt > 0) m = (cnt & 1) ? v[cnt / 2] : 0.5f * (v[cnt / 2 - 1] + v[cnt / 2]);
    out[p] = m;
  }
}

sfft_status_t fail(cudaError_t e, const char* where) {
  sfft::set_last_error((std::string(where) + ": " + cudaGetErrorString(e)).c_str());
  return SFFT_ERR_CUDA;
}

bool args_ok(int32_t H, int32_t W, int32_t batch, const float* D, const double* pos, int32_t n, double radius) {
  return H > 0 && W > 0 && batch > 0 && D && n >= 0 && (n == 0 || pos) && radius > 0.0 && radius <= 32.0;
}

}  // namespace

extern "C" sfft_status_t phot_aperture_flux(int32_t H, int32_t W, int32_t batch, const float* D, const uint8_t* bad,
                                            const double* pos, int32_t n, double radius, double* flux, int32_t* flag,
                                            void* stream) {
  if (!args_ok(H, W, batch, D, pos, n, radius) || (n > 0 && (!flux || !flag))) return SFFT_ERR_ARG;
  if (n == 0) return SFFT_OK;
  const int64_t items = (int64_t)batch * n;
  k_aperture<<<(unsigned)((items + 7) / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(H, W, batch, D, bad, pos, n,
                                                                                       radius, flux, flag);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : fail(e, "phot_aperture_flux");
}

extern "C" size_t phot_limiting_workspace_bytes(int32_t batch, int32_t n) {
  if (batch < 1 || n < 1) return 0;
  const size_t nb = (size_t)batch * n;
  return ((nb * sizeof(double) + 255) & ~size_t(255)) + nb * sizeof(int32_t);
}

extern "C" sfft_status_t phot_limiting_mag(int32_t H, int32_t W, int32_t batch, const float* D, const uint8_t* bad,
                                           const double* pos, int32_t n, double radius, double zp, double* sigma,
                                           double* mlim, int32_t* ngood, void* ws, void* stream) {
  if (!args_ok(H, W, batch, D, pos, n, radius) || n < 2 || !sigma || !mlim || !ngood || !ws ||
      (reinterpret_cast<uintptr_t>(ws) & 255))
    return SFFT_ERR_ARG;
  const size_t nb = (size_t)batch * n;
  double* flux = static_cast<double*>(ws);
  int32_t* flag = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + ((nb * sizeof(double) + 255) & ~size_t(255)));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_aperture<<<(unsigned)((nb + 7) / 8), 256, 0, s>>>(H, W, batch, D, bad, pos, n, radius, flux, flag);
  k_limit<<<batch, 256, 0, s>>>(flux, flag, n, zp, sigma, mlim, ngood);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : fail(e, "phot_limiting_mag");
}

extern "C" sfft_status_t phot_median_combine(int32_t H, int32_t W, int32_t ntemp, const float* D, const float* scale,
                                             const uint8_t* bad, float* out, void* stream) {
  if (H <= 0 || W <= 0 || ntemp < 1 || !D || !scale || !out) return SFFT_ERR_ARG;
  if (ntemp > kMaxTemplates) return SFFT_ERR_UNSUPPORTED;
  const int64_t npx = (int64_t)H * W;
  const int grid = (int)std::min<int64_t>((npx + 255) / 256, 152 * 16);
  k_median_combine<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(npx, ntemp, D, scale, bad, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : fail(e, "phot_median_combine");
}
