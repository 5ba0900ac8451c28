// Mask and sky-offset preparation, fit-mask erosion and the background
// moments.
//   good(x)  = bad(x) == 0 && finite(R(x)) && finite(S(x))
//   R_m(x)   = good ? R - s_R : 0
//   M_fit(x) = x at least w from every edge and good on the whole L x L
//              footprint (separable erosion: a row pass, then a column pass)
//   moments  sum_x M_fit xt^a yt^b (a + b <= 2 D_B)  and
//            sum_x M_fit xt^a yt^b v(x) (a + b <= D_B), v = S - s_S or the
//            refinement residual e; FP32 per-thread partials, FP64 block and
//            global accumulation.
// The sky constants, when not given, are the mean of the good pixels rounded
// to an integer, so R - s_R and S - s_S are exact in FP32 for |R|, |S| < 2^24.
#include "common.cuh"
#include "plan.h"

namespace sfft {

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
  }
  return s;  // valid on thread 0
}

// block_sum with the warp stage in T (FP32 on the mixed path: GB300 retires
// two FP64 operations per SM per clock, so FP64 shuffle trees in every warp
// dominated the kernels that sum per row) and the warps' sums in FP64
template <int NT, typename T>
__device__ __forceinline__ double block_sum_t(T v, double* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
    s = warp_sum(s);
  }
  return s;  // valid on thread 0
}

// Sums of R, S and the count over the good pixels, per CCD.  Where a CCD's
// images start on 16-byte boundaries the pixels go in groups of four (float4
// and uchar4 loads); the launch gives each thread at most 64 groups, so a
// thread's FP32 partial sums cover at most 256 pixels before the FP64 block
// sums.
__global__ void __launch_bounds__(256)
k_sky_sum(const float* __restrict__ R, const float* __restrict__ S, const uint8_t* __restrict__ bad, int64_t npx,
          double* __restrict__ acc) {
  __shared__ double red[8];
  const int ccd = blockIdx.y;
  const float* r = R + ccd * npx;
  const float* s = S + ccd * npx;
  const uint8_t* b = bad ? bad + ccd * npx : nullptr;
  float sr = 0.f, ss = 0.f;
  int cnt = 0;
  const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(r) | reinterpret_cast<uintptr_t>(s)) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(b) & 3) == 0;
  int64_t i0 = 0;
  if (vec) {
    const int64_t n4 = npx / 4;
    const float4* r4 = reinterpret_cast<const float4*>(r);
    const float4* s4 = reinterpret_cast<const float4*>(s);
    const uchar4* b4 = reinterpret_cast<const uchar4*>(b);
#pragma unroll 4
    for (int64_t q = t0; q < n4; q += nt) {
      const float4 rv = r4[q], sv = s4[q];
      const uchar4 bv = b ? b4[q] : make_uchar4(0, 0, 0, 0);
      const float ra[4] = {rv.x, rv.y, rv.z, rv.w}, sa[4] = {sv.x, sv.y, sv.z, sv.w};
      const unsigned char ba[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (ba[k] == 0 && isfinite(ra[k]) && isfinite(sa[k])) { sr += ra[k]; ss += sa[k]; ++cnt; }
    }
    i0 = n4 * 4;
  }
  for (int64_t i = i0 + t0; i < npx; i += nt) {
    const float rv = r[i], sv = s[i];
    if ((!b || b[i] == 0) && isfinite(rv) && isfinite(sv)) { sr += rv; ss += sv; ++cnt; }
  }
  const double d0 = block_sum<256>((double)sr, red);
  if (threadIdx.x == 0) atomicAdd(&acc[4 * ccd + 0], d0);
  const double d1 = block_sum<256>((double)ss, red);
  if (threadIdx.x == 0) atomicAdd(&acc[4 * ccd + 1], d1);
  const double d2 = block_sum<256>((double)cnt, red);
  if (threadIdx.x == 0) atomicAdd(&acc[4 * ccd + 2], d2);
}

__global__ void k_sky_final(const double* __restrict__ acc, double* __restrict__ sky, int batch) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= batch) return;
  const double n = acc[4 * c + 2];
  sky[2 * c + 0] = n > 0 ? rint(acc[4 * c + 0] / n) : 0.0;
  sky[2 * c + 1] = n > 0 ? rint(acc[4 * c + 1] / n) : 0.0;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_prep(const float* __restrict__ R, const float* __restrict__ S, const uint8_t* __restrict__ bad,
       const double* __restrict__ sky, int64_t npx, uint8_t* __restrict__ good, T* __restrict__ Rm) {
  const int ccd = blockIdx.y;
  const T sR = (T)sky[2 * ccd];
  const int64_t base = ccd * npx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npx; i += (int64_t)gridDim.x * blockDim.x) {
    const float rv = R[base + i], sv = S[base + i];
    const bool g = (!bad || bad[base + i] == 0) && isfinite(rv) && isfinite(sv);
    good[base + i] = g ? 1 : 0;
    Rm[base + i] = g ? (T)rv - sR : (T)0;
  }
}

// row pass: gh(y, x) = w <= x < W - w and good on [x - w, x + w]
__global__ void __launch_bounds__(256)
k_erode_rows(const uint8_t* __restrict__ good, uint8_t* __restrict__ gh, int H, int W, int w) {
  const int y = blockIdx.x, ccd = blockIdx.y;
  const uint8_t* g = good + ((int64_t)ccd * H + y) * W;
  uint8_t* o = gh + ((int64_t)ccd * H + y) * W;
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    uint8_t v = 0;
    if (x >= w && x < W - w) {
      v = 1;
      for (int dx = -w; dx <= w; ++dx) v &= g[x + dx];
    }
    o[x] = v;
  }
}

// column pass: M(y, x) = w <= y < H - w and gh on [y - w, y + w]
__global__ void __launch_bounds__(256)
k_erode_cols(const uint8_t* __restrict__ gh, uint8_t* __restrict__ mfit, int H, int W, int w) {
  const int y = blockIdx.x, ccd = blockIdx.y;
  const uint8_t* g = gh + (int64_t)ccd * H * W;
  uint8_t* o = mfit + ((int64_t)ccd * H + y) * W;
  const bool inside = (y >= w && y < H - w);
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    uint8_t v = 0;
    if (inside) {
      v = 1;
      for (int dy = -w; dy <= w; ++dy) v &= g[(int64_t)(y + dy) * W + x];
    }
    o[x] = v;
  }
}

// one block per (row, ccd).  mom_bb[mono(a,b)] for a+b <= DBB, mom_v[mono(a,b)] for a+b <= DV.
// Per CCD the background moments sum_x M_fit xt^a yt^b (a + b <= DBB) and
// sum_x M_fit xt^a yt^b v(x) (a + b <= DV), with yt^b factored out of each
// row.  A CTA takes kMomRows consecutive rows, a warp per row at a time.  A
// lane sums its pixels in groups of four (float4 / uchar4 loads where the row
// is 16-byte aligned): each group's sum in T, added to the lane's T sums, then
// a warp tree in T gives the row's sums.  The row's FP64 contributions are
// added over the CTA's rows (fixed order) and then atomically to the CCD's
// moments, so each moment takes H / kMomRows atomic adds per CCD instead of H.
constexpr int kMomRows = 8;

template <typename T>
__device__ __forceinline__ void load4(const T* p, T (&v)[4]);
template <>
__device__ __forceinline__ void load4<float>(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void load4<double>(const double* p, double (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_moments(const uint8_t* __restrict__ mfit, const float* __restrict__ S, const double* __restrict__ sky,
          const T* __restrict__ E, int H, int W, int DBB, int DV, double* __restrict__ mom_bb, int64_t bb_stride,
          double* __restrict__ mom_v, int64_t v_stride, int* __restrict__ rowflag, int rf_stride) {
  constexpr int NBB = n_mono(kMaxWeightDeg), NV = n_mono(kMaxD);
  __shared__ double part[8][NBB + NV];
  const int ccd = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T sS = S ? (T)sky[2 * ccd + 1] : (T)0;
  const T xs = (T)2 / (T)(W > 1 ? W - 1 : 1);
  const double ysc = 2.0 / (double)(H > 1 ? H - 1 : 1);
  // part[w]: warp w's rows, FP64, added to by its lane 0
  for (int i = threadIdx.x; i < 8 * (NBB + NV); i += blockDim.x) (&part[0][0])[i] = 0.0;
  __syncthreads();
  const int y_end = min(H, ((int)blockIdx.x + 1) * kMomRows);
  for (int y = (int)blockIdx.x * kMomRows + warp; y < y_end; y += 8) {
    const int64_t row = ((int64_t)ccd * H + y) * W;
    const uint8_t* mr = mfit + row;
    const float* sr = S ? S + row : nullptr;
    const T* er = E ? E + row : nullptr;
    T pm[kMaxWeightDeg + 1] = {0, 0, 0, 0, 0};
    T pv[kMaxD + 1] = {0, 0, 0};
    int cnt = 0;
    // adds the pixels of one group (mk: in the fit mask, vk: S - s_S or e)
    auto add_group = [&](const int x0, const bool (&mk)[4], const T (&vk)[4], int n) {
      T gm[kMaxWeightDeg + 1] = {0, 0, 0, 0, 0};
      T gv[kMaxD + 1] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k >= n || !mk[k]) continue;
        ++cnt;
        const T xt = (T)(x0 + k) * xs - (T)1;
        T pw = 1;
#pragma unroll
        for (int a = 0; a <= kMaxWeightDeg; ++a) {
          gm[a] += pw;
          if (a <= kMaxD) gv[a] += pw * vk[k];
          pw *= xt;
        }
      }
#pragma unroll
      for (int a = 0; a <= kMaxWeightDeg; ++a) pm[a] += gm[a];
#pragma unroll
      for (int a = 0; a <= kMaxD; ++a) pv[a] += gv[a];
    };
    const bool vec = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(mr) & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(sr) & 15) == 0 && (reinterpret_cast<uintptr_t>(er) & 15) == 0;
    if (vec) {
#pragma unroll 4
      for (int x0 = 4 * lane; x0 < W; x0 += 128) {
        const uchar4 m4 = *reinterpret_cast<const uchar4*>(mr + x0);
        const bool mk[4] = {m4.x != 0, m4.y != 0, m4.z != 0, m4.w != 0};
        T vk[4] = {0, 0, 0, 0};
        if (sr) {
          float f[4];
          load4<float>(sr + x0, f);
#pragma unroll
          for (int k = 0; k < 4; ++k) vk[k] = (T)f[k] - sS;
        } else if (er) {
          load4<T>(er + x0, vk);
        }
        add_group(x0, mk, vk, 4);
      }
    } else {
      for (int x0 = 4 * lane; x0 < W; x0 += 128) {
        const int n = min(4, W - x0);
        bool mk[4];
        T vk[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          mk[k] = k < n && mr[x0 + k] != 0;
          vk[k] = k < n ? (sr ? (T)sr[x0 + k] - sS : (er ? er[x0 + k] : (T)0)) : (T)0;
        }
        add_group(x0, mk, vk, n);
      }
    }
    cnt = warp_sum(cnt);
#pragma unroll
    for (int a = 0; a <= kMaxWeightDeg; ++a) pm[a] = warp_sum(pm[a]);
#pragma unroll
    for (int a = 0; a <= kMaxD; ++a) pv[a] = warp_sum(pv[a]);
    if (lane == 0) {
      if (rowflag) rowflag[(int64_t)ccd * rf_stride + y] = cnt > 0 ? 1 : 0;
      const double yt = (double)y * ysc - 1.0;
#pragma unroll
      for (int a = 0; a <= kMaxWeightDeg; ++a) {
        double yp = 1.0;
#pragma unroll
        for (int b = 0; a + b <= kMaxWeightDeg; ++b) {
          if (a + b <= DBB) part[warp][mono_index(a, b)] += (double)pm[a] * yp;
          yp *= yt;
        }
      }
#pragma unroll
      for (int a = 0; a <= kMaxD; ++a) {
        double yp = 1.0;
#pragma unroll
        for (int b = 0; a + b <= kMaxD; ++b) {
          if (a + b <= DV) part[warp][NBB + mono_index(a, b)] += (double)pv[a] * yp;
          yp *= yt;
        }
      }
    }
  }
  __syncthreads();
  const int nbb = mom_bb ? n_mono(DBB) : 0, nv = n_mono(DV);
  if (threadIdx.x < nbb + nv) {
    const int i = threadIdx.x < nbb ? threadIdx.x : NBB + (threadIdx.x - nbb);
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += part[w][i];
    if (threadIdx.x < nbb) atomicAdd(&mom_bb[ccd * bb_stride + threadIdx.x], s);
    else atomicAdd(&mom_v[ccd * v_stride + (threadIdx.x - nbb)], s);
  }
}

static int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  return (int)(g < cap ? (g < 1 ? 1 : g) : cap);
}

cudaError_t launch_sky(const sfft_plan_s* p, const float* R, const float* S, const uint8_t* bad,
                       const double* sky_in, void* ws) {
  double* sky = ws_at<double>(ws, p->sky);
  const int B = p->d.batch;
  if (sky_in) {
    return cudaMemcpyAsync(sky, sky_in, sizeof(double) * 2 * B, cudaMemcpyDeviceToDevice, p->stream);
  }
  double* acc = ws_at<double>(ws, p->skyacc);
  cudaMemsetAsync(acc, 0, sizeof(double) * 4 * B, p->stream);
  const int64_t npx = (int64_t)p->d.H * p->d.W;
  // at least four CTAs per SM, and at most 64 groups of four pixels per thread
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t per_cta = 256 * 64 * 4;
  const int gx = (int)std::min<int64_t>(std::max<int64_t>(4 * (int64_t)std::max(sms, 1), (npx + per_cta - 1) / per_cta),
                                        1 << 20);
  k_sky_sum<<<dim3(gx, B), 256, 0, p->stream>>>(R, S, bad, npx, acc);
  k_sky_final<<<(B + 127) / 128, 128, 0, p->stream>>>(acc, sky, B);
  p->nlaunch += 2;
  return cudaGetLastError();
}

template <typename T>
static cudaError_t prep_T(const sfft_plan_s* p, const float* R, const float* S, const uint8_t* bad, void* ws) {
  const int H = p->d.H, W = p->d.W, B = p->d.batch;
  const int64_t npx = (int64_t)H * W;
  uint8_t* good = ws_at<uint8_t>(ws, p->good);
  uint8_t* gh = ws_at<uint8_t>(ws, p->gh);
  uint8_t* mfit = ws_at<uint8_t>(ws, p->mfit);
  T* Rm = ws_at<T>(ws, p->rm);
  dim3 g1(grid_for(npx, 256 * 8, 1184), B);
  k_prep<T><<<g1, 256, 0, p->stream>>>(R, S, bad, ws_at<double>(ws, p->sky), npx, good, Rm);
  dim3 g2(H, B);
  k_erode_rows<<<g2, 256, 0, p->stream>>>(good, gh, H, W, p->w);
  k_erode_cols<<<g2, 256, 0, p->stream>>>(gh, mfit, H, W, p->w);
  p->nlaunch += 3;
  return cudaGetLastError();
}

cudaError_t launch_prep(const sfft_plan_s* p, const float* R, const float* S, const uint8_t* bad, void* ws) {
  return p->fp64 ? prep_T<double>(p, R, S, bad, ws) : prep_T<float>(p, R, S, bad, ws);
}

// resid == false: BB moments, b_B (from S) and row flags;  resid == true: b_B-part of the
// refinement right-hand side from the residual image (written into vec slot 0 tail).
template <typename T>
static cudaError_t moments_T(const sfft_plan_s* p, const float* S, const void* eimg, bool resid, void* ws) {
  const int H = p->d.H, W = p->d.W, B = p->d.batch;
  const uint8_t* mfit = ws_at<uint8_t>(ws, p->mfit);
  const double* sky = ws_at<double>(ws, p->sky);
  dim3 g((H + kMomRows - 1) / kMomRows, B);
  if (!resid) {
    double* bb = ws_at<double>(ws, p->mom_bb);
    double* bv = ws_at<double>(ws, p->mom_b);
    const int nbb = n_mono(p->DM_BB), nb = n_mono(p->d.DB);
    cudaMemsetAsync(bb, 0, sizeof(double) * nbb * B, p->stream);
    cudaMemsetAsync(bv, 0, sizeof(double) * nb * B, p->stream);
    k_moments<T><<<g, 256, 0, p->stream>>>(mfit, S, sky, (const T*)nullptr, H, W, p->DM_BB, p->d.DB, bb, nbb, bv,
                                           nb, ws_at<int>(ws, p->rowflag), p->rf_stride);
  } else {
    double* bv = ws_at<double>(ws, p->mom_b);
    const int nb = n_mono(p->d.DB);
    cudaMemsetAsync(bv, 0, sizeof(double) * nb * B, p->stream);
    k_moments<T><<<g, 256, 0, p->stream>>>(mfit, nullptr, sky, (const T*)eimg, H, W, 0, p->d.DB, nullptr, 0, bv,
                                           nb, nullptr, 0);
  }
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_moments(const sfft_plan_s* p, const float* S, const void* eimg, bool resid, void* ws) {
  return p->fp64 ? moments_T<double>(p, S, eimg, resid, ws) : moments_T<float>(p, S, eimg, resid, ws);
}

}  // namespace sfft
