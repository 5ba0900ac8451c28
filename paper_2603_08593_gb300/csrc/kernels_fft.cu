// Batched real-to-complex row FFTs with shared-memory staging (one warp per
// image row).  Row length Nf = 2M (power of two, 64..2048, zero padded past
// W).  The real row x[n] is packed as z[n] = x[2n] + i x[2n+1] (M points),
// transformed by a two-pass M = 32 * N2 decomposition (a length-N2 DFT in
// registers over n2, twiddle exp(-2 pi i n1 k2 / M), a padded shared-memory
// transpose, a length-32 DFT in registers over n1), then split into the
// real-input spectrum X[k], k = 0..M.  Output row layout: M complex slots,
// slot 0 packs the two real bins (X[0], X[M]); slot k holds X[k] otherwise.
//
// Three row sources feed the same transform:
//   products   P_d(y, x) = R_m(y, x) R_m(y + d_y, x + d_x)   (zero off-image)
//   reference  R_m(y, x)
//   weights    M_fit(y, x) xt^a [ * (S(y, x) - s_S) | * e(y, x) ]
#include "common.cuh"
#include "plan.h"

namespace sfft {

template <typename T> constexpr int fft_warps() { return sizeof(T) == 4 ? 8 : 4; }
template <typename T> __host__ __device__ constexpr int fft_smem_per_warp() { return 2 * 1056 * (int)sizeof(T); }

// z (registers, lane n1 holds z[n1 + 32 n2] in z[n2]) -> packed spectrum row `out`.
// The shared-memory pointers must not be __restrict__: lanes read back slots
// that other lanes rewrote after the __syncwarp, and a restrict qualifier lets
// the compiler forward a lane's own earlier store instead of reloading.
template <typename T, int N2>
__device__ __forceinline__ void warp_rfft(c_t<T> (&z)[N2], T* sre, T* sim,
                                          const c_t<T>* __restrict__ twM, const c_t<T>* __restrict__ twN,
                                          c_t<T>* __restrict__ out) {
  using T2 = c_t<T>;
  constexpr int M = 32 * N2;
  const int lane = threadIdx.x & 31;
  fft_reg<N2>(z);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) {
    T2 v = cmul(z[k2], twM[k2 * 32 + lane]);
    sre[k2 * 33 + lane] = v.x;
    sim[k2 * 33 + lane] = v.y;
  }
  __syncwarp();
  T2 v[32];
  if (lane < N2) {
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) { v[n1].x = sre[lane * 33 + n1]; v[n1].y = sim[lane * 33 + n1]; }
    fft_reg<32>(v);
  }
  __syncwarp();
  if (lane < N2) {
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) { sre[lane + N2 * k1] = v[k1].x; sim[lane + N2 * k1] = v[k1].y; }
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < N2; ++t) {
    const int k = lane + 32 * t;
    const int km = (M - k) & (M - 1);
    const T zr = sre[k], zi = sim[k], mr = sre[km], mi = sim[km];
    T2 X;
    if (k == 0) {
      X.x = zr + zi;
      X.y = zr - zi;
    } else {
      const T er = (T)0.5 * (zr + mr), ei = (T)0.5 * (zi - mi);
      const T orr = (T)0.5 * (zr - mr), oi = (T)0.5 * (zi + mi);
      const T2 wk = twN[k];
      const T wr = wk.x * orr - wk.y * oi, wi = wk.x * oi + wk.y * orr;
      X.x = er + wi;
      X.y = ei - wr;
    }
    out[k] = X;
  }
  __syncwarp();
}

// products (self == 0) or the plain R_m spectrum (self == 1)
template <typename T, int N2>
__global__ void __launch_bounds__(32 * fft_warps<T>())
k_rfft_prod(const T* __restrict__ Rm, int H, int W, const int2* __restrict__ dl, int d0, int self,
            c_t<T>* __restrict__ out, int64_t slab_stride, int64_t ccd_stride_out,
            const c_t<T>* __restrict__ twM, const c_t<T>* __restrict__ twN) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int M = 32 * N2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* sre = reinterpret_cast<T*>(smem_raw + warp * fft_smem_per_warp<T>());
  T* sim = sre + 1056;
  const int jd = blockIdx.y, ccd = blockIdx.z;
  int dy = 0, dx = 0;
  if (!self) { const int2 dd = dl[d0 + jd]; dy = dd.x; dx = dd.y; }
  const T* img = Rm + (int64_t)ccd * H * W;
  c_t<T>* obase = out + (int64_t)ccd * ccd_stride_out + (int64_t)jd * slab_stride;
  for (int y = blockIdx.x * fft_warps<T>() + warp; y < H; y += gridDim.x * fft_warps<T>()) {
    const T* row = img + (int64_t)y * W;
    const bool ok2 = (y + dy >= 0) && (y + dy < H);
    const T* row2 = img + (int64_t)(y + dy) * W;
    c_t<T> z[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      const int x0 = 2 * (lane + 32 * n2), x1 = x0 + 1;
      T v0 = x0 < W ? row[x0] : (T)0;
      T v1 = x1 < W ? row[x1] : (T)0;
      if (!self) {
        const int s0 = x0 + dx, s1 = x1 + dx;
        v0 *= (ok2 && s0 >= 0 && s0 < W) ? row2[s0] : (T)0;
        v1 *= (ok2 && s1 >= 0 && s1 < W) ? row2[s1] : (T)0;
      }
      z[n2].x = v0;
      z[n2].y = v1;
    }
    warp_rfft<T, N2>(z, sre, sim, twM, twN, obase + (int64_t)y * M);
  }
}

// weights M_fit xt^a, optionally times (S - s_S) (S != null) or e (E != null)
template <typename T, int N2>
__global__ void __launch_bounds__(32 * fft_warps<T>())
k_rfft_weight(const uint8_t* __restrict__ Mfit, const float* __restrict__ S, const double* __restrict__ sky,
              const T* __restrict__ E, int H, int W, int a0, c_t<T>* __restrict__ out, int64_t slab_stride,
              int64_t ccd_stride_out, const c_t<T>* __restrict__ twM, const c_t<T>* __restrict__ twN) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int M = 32 * N2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* sre = reinterpret_cast<T*>(smem_raw + warp * fft_smem_per_warp<T>());
  T* sim = sre + 1056;
  const int a = a0 + blockIdx.y, ccd = blockIdx.z;
  const int64_t img_off = (int64_t)ccd * H * W;
  const T sS = S ? (T)sky[2 * ccd + 1] : (T)0;
  const T xs = (T)2.0 / (T)(W > 1 ? W - 1 : 1);
  c_t<T>* obase = out + (int64_t)ccd * ccd_stride_out + (int64_t)blockIdx.y * slab_stride;
  for (int y = blockIdx.x * fft_warps<T>() + warp; y < H; y += gridDim.x * fft_warps<T>()) {
    const uint8_t* mrow = Mfit + img_off + (int64_t)y * W;
    c_t<T> z[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      T v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int x = 2 * (lane + 32 * n2) + h;
        T val = (T)0;
        if (x < W && mrow[x]) {
          const T xt = (T)x * xs - (T)1;
          T pw = (T)1;
          for (int i = 0; i < a; ++i) pw *= xt;
          if (S) pw *= ((T)S[img_off + (int64_t)y * W + x] - sS);
          else if (E) pw *= E[img_off + (int64_t)y * W + x];
          val = pw;
        }
        v[h] = val;
      }
      z[n2].x = v[0];
      z[n2].y = v[1];
    }
    warp_rfft<T, N2>(z, sre, sim, twM, twN, obase + (int64_t)y * M);
  }
}

template <typename T, int N2>
static cudaError_t run_prod(const sfft_plan_s* p, const T* Rm, int d0, int nd, int self, c_t<T>* out,
                            int64_t slab_stride, int64_t ccd_stride) {
  const int warps = fft_warps<T>();
  const size_t smem = (size_t)warps * fft_smem_per_warp<T>();
  auto kern = k_rfft_prod<T, N2>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int H = p->d.H;
  int gx = (H + warps - 1) / warps;
  dim3 grid(gx, self ? 1 : nd, p->d.batch);
  kern<<<grid, 32 * warps, smem, p->stream>>>(Rm, H, p->d.W, p->d_dlist, d0, self, out, slab_stride, ccd_stride,
                                              (const c_t<T>*)p->twM, (const c_t<T>*)p->twN);
  p->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T, int N2>
static cudaError_t run_weight(const sfft_plan_s* p, const uint8_t* Mfit, const float* S, const double* sky,
                              const T* E, int a0, int na, c_t<T>* out, int64_t slab_stride, int64_t ccd_stride) {
  const int warps = fft_warps<T>();
  const size_t smem = (size_t)warps * fft_smem_per_warp<T>();
  auto kern = k_rfft_weight<T, N2>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int H = p->d.H;
  dim3 grid((H + warps - 1) / warps, na, p->d.batch);
  kern<<<grid, 32 * warps, smem, p->stream>>>(Mfit, S, sky, E, H, p->d.W, a0, out, slab_stride, ccd_stride,
                                              (const c_t<T>*)p->twM, (const c_t<T>*)p->twN);
  p->nlaunch += 1;
  return cudaGetLastError();
}

#define SFFT_DISPATCH_N2(N2V, CALL) \
  switch (N2V) {                    \
    case 1: { constexpr int N2 = 1; return CALL; } \
    case 2: { constexpr int N2 = 2; return CALL; } \
    case 4: { constexpr int N2 = 4; return CALL; } \
    case 8: { constexpr int N2 = 8; return CALL; } \
    case 16: { constexpr int N2 = 16; return CALL; } \
    case 32: { constexpr int N2 = 32; return CALL; } \
    default: return cudaErrorInvalidValue; \
  }

template <typename T>
static cudaError_t prod_T(const sfft_plan_s* p, int d0, int nd, void* ws) {
  const int64_t HM = (int64_t)p->d.H * p->M;
  const T* Rm = ws_at<T>(ws, p->rm);
  c_t<T>* out = ws_at<c_t<T>>(ws, p->phat);
  SFFT_DISPATCH_N2(p->N2, (run_prod<T, N2>(p, Rm, d0, nd, 0, out, HM, HM * p->d_batch)))
}

template <typename T>
static cudaError_t rm_T(const sfft_plan_s* p, void* ws) {
  const int64_t HM = (int64_t)p->d.H * p->M;
  const T* Rm = ws_at<T>(ws, p->rm);
  c_t<T>* out = ws_at<c_t<T>>(ws, p->rhat);
  SFFT_DISPATCH_N2(p->N2, (run_prod<T, N2>(p, Rm, 0, 1, 1, out, HM, HM)))
}

template <typename T>
static cudaError_t weights_T(const sfft_plan_s* p, const float* S, const void* eimg, int a0, int na, void* out,
                             int nslab, void* ws) {
  // `out` is the base of a region holding `nslab` spectra per CCD; slabs a0 .. a0+na-1 are written
  const int64_t HM = (int64_t)p->d.H * p->M;
  const uint8_t* Mfit = ws_at<uint8_t>(ws, p->mfit);
  const double* sky = ws_at<double>(ws, p->sky);
  SFFT_DISPATCH_N2(p->N2, (run_weight<T, N2>(p, Mfit, S, sky, (const T*)eimg, a0, na,
                                             (c_t<T>*)out + a0 * HM, HM, HM * nslab)))
}

cudaError_t launch_rfft_prod(const sfft_plan_s* p, int d0, int nd, void* ws) {
  return p->fp64 ? prod_T<double>(p, d0, nd, ws) : prod_T<float>(p, d0, nd, ws);
}
cudaError_t launch_rfft_rm(const sfft_plan_s* p, void* ws) {
  return p->fp64 ? rm_T<double>(p, ws) : rm_T<float>(p, ws);
}
cudaError_t launch_rfft_weights(const sfft_plan_s* p, const float* S, const void* eimg, int a0, int na, void* out,
                                int nslab, void* ws) {
  return p->fp64 ? weights_T<double>(p, S, eimg, a0, na, out, nslab, ws)
                 : weights_T<float>(p, S, eimg, a0, na, out, nslab, ws);
}

}  // namespace sfft
