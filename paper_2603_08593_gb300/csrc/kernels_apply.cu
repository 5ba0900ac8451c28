// Spatially varying convolution and subtraction (and the refinement residual).
//
//   model(x) = sum_p phi_p(x) sum_j theta[j, p] R~(x - u_j) + B'(x),
//   R~ = finite(R) ? R - s_R : 0, zero outside the image;
//   D(x) = S(x) - s_S - model(x)                       (apply)
//   e(x) = M_fit(x) ? S(x) - s_S - model(x) : 0        (refinement residual)
//
// A CTA covers a 64 x 32 output tile and stages the (64 + 2w) x (32 + 2w)
// halo of R~ and the L^2 N_K coefficients in shared memory; each thread keeps
// the N_K partial convolutions of 8 vertically adjacent pixels in registers
// and slides down the staged column, so every shared-memory value feeds
// 8 N_K fused multiply-adds.
#include "common.cuh"
#include "plan.h"

namespace sfft {

constexpr int AP_TX = 32, AP_TY = 64, AP_RY = 8;   // tile, rows per thread
constexpr int AP_THREADS = AP_TX * (AP_TY / AP_RY); // 256

template <typename T, int NK, bool RESID>
__global__ void __launch_bounds__(AP_THREADS)
k_apply(const float* __restrict__ R, const float* __restrict__ S, const double* __restrict__ theta_off,
        const double* __restrict__ sky, const uint8_t* __restrict__ mfit, float* __restrict__ D, T* __restrict__ E,
        int H, int W, int L, int DB) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int w = (L - 1) / 2;
  const int LL = L * L;
  const int NB = n_mono(DB);
  const int N = LL * NK + NB;
  const int tw = AP_TX + 2 * w, th = AP_TY + 2 * w;
  T* coef = reinterpret_cast<T*>(smraw);           // [LL][NK]
  T* beta = coef + LL * NK;                         // [NB]
  T* tile = beta + 8;                               // [th][tw]
  const int ccd = blockIdx.z;
  const int64_t img = (int64_t)ccd * H * W;
  const double* th_c = theta_off + (int64_t)ccd * N;
  for (int i = threadIdx.x; i < LL * NK; i += blockDim.x) coef[i] = (T)th_c[i];
  for (int i = threadIdx.x; i < NB; i += blockDim.x) beta[i] = (T)th_c[LL * NK + i];
  const T sR = (T)sky[2 * ccd], sS = (T)sky[2 * ccd + 1];
  const int x0 = blockIdx.x * AP_TX, y0 = blockIdx.y * AP_TY;
  for (int i = threadIdx.x; i < th * tw; i += blockDim.x) {
    const int ty = i / tw, tx = i % tw;
    const int gy = y0 - w + ty, gx = x0 - w + tx;
    T v = 0;
    if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
      const float r = R[img + (int64_t)gy * W + gx];
      v = isfinite(r) ? (T)r - sR : (T)0;
    }
    tile[i] = v;
  }
  __syncthreads();
  const int tx = threadIdx.x % AP_TX, tyb = (threadIdx.x / AP_TX) * AP_RY;
  const int gx = x0 + tx;
  T acc[AP_RY][NK];
#pragma unroll
  for (int r = 0; r < AP_RY; ++r)
#pragma unroll
    for (int p = 0; p < NK; ++p) acc[r][p] = 0;
  for (int uy = -w; uy <= w; ++uy) {
    for (int ux = -w; ux <= w; ++ux) {
      const int j = (uy + w) * L + (ux + w);
      T c[NK];
#pragma unroll
      for (int p = 0; p < NK; ++p) c[p] = coef[j * NK + p];
      // output row (tyb + r) reads tile row (tyb + r - uy + w), column (tx - ux + w)
      const T* col = tile + (tyb - uy + w) * tw + (tx - ux + w);
#pragma unroll
      for (int r = 0; r < AP_RY; ++r) {
        const T v = col[r * tw];
#pragma unroll
        for (int p = 0; p < NK; ++p) acc[r][p] += c[p] * v;
      }
    }
  }
  if (gx >= W) return;
  const T xs = (T)2 / (T)(W > 1 ? W - 1 : 1), ysc = (T)2 / (T)(H > 1 ? H - 1 : 1);
  const T xt = (T)gx * xs - (T)1;
#pragma unroll
  for (int r = 0; r < AP_RY; ++r) {
    const int gy = y0 + tyb + r;
    if (gy >= H) break;
    const T yt = (T)gy * ysc - (T)1;
    // phi_p / psi_q: degree-major, a descending
    T mono[6];
    mono[0] = 1; mono[1] = xt; mono[2] = yt; mono[3] = xt * xt; mono[4] = xt * yt; mono[5] = yt * yt;
    T model = 0;
#pragma unroll
    for (int p = 0; p < NK; ++p) model += mono[p] * acc[r][p];
    for (int q = 0; q < NB; ++q) model += beta[q] * mono[q];
    const int64_t o = img + (int64_t)gy * W + gx;
    const T sp = (T)S[o] - sS;
    const T dv = sp - model;
    if constexpr (RESID) {
      E[o] = mfit[o] ? dv : (T)0;
    } else {
      D[o] = (float)dv;
    }
  }
}

template <typename T, int NK, bool RESID>
static cudaError_t run_apply(const sfft_plan_s* p, const float* R, const float* S, const double* theta_off,
                             const double* sky, const uint8_t* mfit, float* D, T* E) {
  const int L = p->d.L, w = p->w;
  const size_t smem = sizeof(T) * ((size_t)L * L * NK + 8 + (size_t)(AP_TY + 2 * w) * (AP_TX + 2 * w));
  auto kern = k_apply<T, NK, RESID>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((p->d.W + AP_TX - 1) / AP_TX, (p->d.H + AP_TY - 1) / AP_TY, p->d.batch);
  kern<<<grid, AP_THREADS, smem, p->stream>>>(R, S, theta_off, sky, mfit, D, E, p->d.H, p->d.W, L, p->d.DB);
  p->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T, bool RESID>
static cudaError_t apply_nk(const sfft_plan_s* p, const float* R, const float* S, const double* theta_off,
                            const double* sky, const uint8_t* mfit, float* D, T* E) {
  switch (p->NK) {
    case 1: return run_apply<T, 1, RESID>(p, R, S, theta_off, sky, mfit, D, E);
    case 3: return run_apply<T, 3, RESID>(p, R, S, theta_off, sky, mfit, D, E);
    case 6: return run_apply<T, 6, RESID>(p, R, S, theta_off, sky, mfit, D, E);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int NK>
static cudaError_t run_apply_raw(cudaStream_t s, const float* R, const float* S, const double* theta_off,
                                 const double* sky, float* D, int H, int W, int L, int DB, int batch) {
  const int w = (L - 1) / 2;
  const size_t smem = sizeof(T) * ((size_t)L * L * NK + 8 + (size_t)(AP_TY + 2 * w) * (AP_TX + 2 * w));
  auto kern = k_apply<T, NK, false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((W + AP_TX - 1) / AP_TX, (H + AP_TY - 1) / AP_TY, batch);
  kern<<<grid, AP_THREADS, smem, s>>>(R, S, theta_off, sky, nullptr, D, (T*)nullptr, H, W, L, DB);
  return cudaGetLastError();
}

cudaError_t launch_apply_raw(cudaStream_t s, bool fp64, const float* R, const float* S, const double* theta_off,
                             const double* sky, float* D, int H, int W, int L, int DK, int DB, int batch) {
  const int NK = n_mono(DK);
#define SFFT_APPLY_RAW(T)                                                                                   \
  switch (NK) {                                                                                             \
    case 1: return run_apply_raw<T, 1>(s, R, S, theta_off, sky, D, H, W, L, DB, batch);                     \
    case 3: return run_apply_raw<T, 3>(s, R, S, theta_off, sky, D, H, W, L, DB, batch);                     \
    case 6: return run_apply_raw<T, 6>(s, R, S, theta_off, sky, D, H, W, L, DB, batch);                     \
    default: return cudaErrorInvalidValue;                                                                  \
  }
  if (fp64) { SFFT_APPLY_RAW(double) }
  SFFT_APPLY_RAW(float)
#undef SFFT_APPLY_RAW
}

cudaError_t launch_apply(const sfft_plan_s* p, const float* R, const float* S, const double* theta_off,
                         const double* sky, float* D, void* eimg, bool resid, void* ws) {
  const uint8_t* mfit = ws_at<uint8_t>(ws, p->mfit);
  const double* sk = sky ? sky : ws_at<double>(ws, p->sky);
  if (p->fp64) {
    return resid ? apply_nk<double, true>(p, R, S, theta_off, sk, mfit, D, (double*)eimg)
                 : apply_nk<double, false>(p, R, S, theta_off, sk, mfit, D, (double*)eimg);
  }
  return resid ? apply_nk<float, true>(p, R, S, theta_off, sk, mfit, D, (float*)eimg)
               : apply_nk<float, false>(p, R, S, theta_off, sk, mfit, D, (float*)eimg);
}

}  // namespace sfft
