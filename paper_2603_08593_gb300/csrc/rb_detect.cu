// Candidate detection on difference images and the plain SNR/shape cuts.
//
// Per CCD: four passes of FP64 clipped statistics over the interior (pass 0
// unclipped, passes 1-3 clipped at 3 RMS about the previous pass's mean), a
// separable FP32 Gaussian matched filter (rows, then columns with the
// 1 / (sigma_D ||G||) scale folded in), a 5 x 5 local-maximum test counted per
// row, an exclusive scan over rows and an ordered compaction that writes the
// candidates in row-major order, then a stamp gather.  Block partials of the
// statistics are reduced in a fixed order, so results are deterministic.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "plan.h"
#include "rb.h"

namespace {

constexpr int kMargin = 15, kHalf = 15, kNms = 2, kMaxR = 15;
constexpr int kStatBlocks = 128, kStatPasses = 4;
constexpr double kClipNsig = 3.0, kClipVarShare = 0.97334;

struct Taps {
  float g[2 * kMaxR + 1];
  int r;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct DetectLayout {
  size_t snr, tmp, guard, part, rowcnt, rowoff, total;
  DetectLayout(int H, int W, int B) {
    const size_t img = (size_t)B * H * W * sizeof(float);
    snr = 0;
    tmp = snr + align256(img);
    guard = tmp + align256(img);
    part = guard + align256((size_t)B * H * W);
    rowcnt = part + align256((size_t)B * kStatPasses * (kStatBlocks * 3 + 1) * sizeof(double));
    rowoff = rowcnt + align256((size_t)B * H * sizeof(int));
    total = rowoff + align256((size_t)B * H * sizeof(int));
  }
};

__device__ __forceinline__ bool good_px(const uint8_t* bad, int64_t i) { return bad == nullptr || bad[i] == 0; }

// Per CCD and pass: kStatBlocks block partials (n, sum(x - shift),
// sum((x - shift)^2)) followed by the shift the pass accumulated about.
constexpr int kPassStride = kStatBlocks * 3 + 1;

// Mean and variance of one pass from its partials, summed in a fixed order.
__device__ void pass_moments(const double* pp, double& mean, double& var) {
  __shared__ double red[3][kStatBlocks / 32];
  const int t = threadIdx.x;
  double v[3] = {0.0, 0.0, 0.0};
  if (t < kStatBlocks)
    for (int q = 0; q < 3; ++q) v[q] = pp[t * 3 + q];
  for (int q = 0; q < 3; ++q) v[q] = sfft::warp_sum(v[q]);
  if (t < kStatBlocks && (t & 31) == 0)
    for (int q = 0; q < 3; ++q) red[q][t >> 5] = v[q];
  __syncthreads();
  double acc[3];
  for (int q = 0; q < 3; ++q) {
    double s = 0.0;
    for (int w = 0; w < kStatBlocks / 32; ++w) s += red[q][w];
    acc[q] = s;
  }
  __syncthreads();
  const double m1 = acc[1] / acc[0];
  mean = pp[kStatBlocks * 3] + m1;
  var = acc[2] / acc[0] - m1 * m1;
}

// One statistics pass.  Pass p > 0 keeps |x - mean_{p-1}| <= 3 sqrt(var_{p-1})
// and accumulates about mean_{p-1}; pass 0 keeps every pixel, about 0.
__global__ void __launch_bounds__(256)
k_clip_pass(int H, int W, const float* __restrict__ D, const uint8_t* __restrict__ bad, double* __restrict__ part,
            int pass) {
  const int b = blockIdx.y;
  const int64_t img = (int64_t)H * W;
  const float* Db = D + b * img;
  const uint8_t* bb = bad ? bad + b * img : nullptr;
  double* pb = part + (int64_t)b * kStatPasses * kPassStride;
  double shift = 0.0, thr = INFINITY;
  if (pass > 0) {
    double mean, var;
    pass_moments(pb + (pass - 1) * kPassStride, mean, var);
    shift = mean;
    thr = kClipNsig * sqrt(var);
  }
  const int iw = W - 2 * kMargin, ih = H - 2 * kMargin;
  const int64_t n_in = (int64_t)iw * ih;
  double c = 0.0, s1 = 0.0, s2 = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_in; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (int64_t)(kMargin + k / iw) * W + kMargin + k % iw;
    const float x = Db[i];
    if (!isfinite(x) || !good_px(bb, i)) continue;
    const double d = (double)x - shift;
    if (!(fabs(d) <= thr)) continue;
    c += 1.0;
    s1 += d;
    s2 += d * d;
  }
  __shared__ double red[3][8];
  double v[3] = {c, s1, s2};
  for (int q = 0; q < 3; ++q) v[q] = sfft::warp_sum(v[q]);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 3; ++q) red[q][threadIdx.x >> 5] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 3; ++q) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[q][w];
      pb[pass * kPassStride + blockIdx.x * 3 + q] = s;
    }
    if (blockIdx.x == 0) pb[pass * kPassStride + kStatBlocks * 3] = shift;
  }
}

__global__ void __launch_bounds__(256)
k_filter_rows(int H, int W, const float* __restrict__ D, const uint8_t* __restrict__ bad, Taps taps,
              float* __restrict__ T) {
  extern __shared__ float row[];
  __shared__ float g[2 * kMaxR + 1];
  const int b = blockIdx.y, r = taps.r;
  if (threadIdx.x <= 2 * r) g[threadIdx.x] = taps.g[threadIdx.x];
  const int64_t img = (int64_t)H * W;
  for (int y = blockIdx.x; y < H; y += gridDim.x) {
    const int64_t base = b * img + (int64_t)y * W;
    for (int i = threadIdx.x; i < W + 2 * r; i += blockDim.x) {
      const int x = i - r;
      float v = 0.f;
      if (x >= 0 && x < W) {
        const float d = D[base + x];
        if (isfinite(d) && (bad == nullptr || bad[base + x] == 0)) v = d;
      }
      row[i] = v;
    }
    __syncthreads();
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
      float s = 0.f;
      for (int k = 0; k <= 2 * r; ++k) s = fmaf(g[k], row[x + k], s);
      T[base + x] = s;
    }
    __syncthreads();
  }
}

constexpr int kColTile = 64;   // output rows per block in the column pass

__global__ void __launch_bounds__(256)
k_filter_cols(int H, int W, const float* __restrict__ T, Taps taps, const double* __restrict__ part,
              float* __restrict__ snr) {
  __shared__ float tile[kColTile + 2 * kMaxR][32];
  __shared__ float g[2 * kMaxR + 1];
  const int b = blockIdx.z, r = taps.r;
  if (threadIdx.x <= 2 * r) g[threadIdx.x] = taps.g[threadIdx.x];
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * kColTile;
  double mean, var;
  pass_moments(part + ((int64_t)b * kStatPasses + kStatPasses - 1) * kPassStride, mean, var);
  float norm = 0.f;
  for (int k = 0; k <= 2 * r; ++k) norm += g[k] * g[k];
  const double sigma = sqrt(var / kClipVarShare);
  const float scale = (float)(1.0 / (sigma * (double)norm));
  const int64_t img = (int64_t)H * W;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int j = ty; j < kColTile + 2 * r; j += 8) {
    const int y = y0 + j - r, x = x0 + tx;
    tile[j][tx] = (y >= 0 && y < H && x < W) ? T[b * img + (int64_t)y * W + x] : 0.f;
  }
  __syncthreads();
  const int x = x0 + tx;
  if (x >= W) return;
  for (int j = ty; j < kColTile; j += 8) {
    const int y = y0 + j;
    if (y >= H) break;
    float s = 0.f;
    for (int k = 0; k <= 2 * r; ++k) s = fmaf(g[k], tile[j + k][tx], s);
    snr[b * img + (int64_t)y * W + x] = s * scale;
  }
}

// bad-pixel guard band, separable: rows then columns (Chebyshev distance <= g)
__global__ void __launch_bounds__(256)
k_dilate_rows(int H, int W, const uint8_t* __restrict__ bad, int g, uint8_t* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)H * W; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = (int64_t)blockIdx.y * H * W;
    const int x = (int)(e % W);
    const int64_t row = base + e - x;
    uint8_t v = 0;
    for (int dx = max(0, x - g); dx <= min(W - 1, x + g); ++dx) v |= bad[row + dx];
    out[base + e] = v ? 1 : 0;
  }
}

__global__ void __launch_bounds__(256)
k_dilate_cols(int H, int W, const uint8_t* __restrict__ in, int g, uint8_t* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)H * W; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = (int64_t)blockIdx.y * H * W;
    const int x = (int)(e % W), y = (int)(e / W);
    uint8_t v = 0;
    for (int dy = max(0, y - g); dy <= min(H - 1, y + g); ++dy) v |= in[base + (int64_t)dy * W + x];
    out[base + e] = v;
  }
}

// candidate predicate; (y, x) inside the margin
__device__ __forceinline__ bool is_candidate(const float* sb, const uint8_t* bb, int W, int y, int x, float thresh) {
  const int64_t i = (int64_t)y * W + x;
  if (bb && bb[i]) return false;
  const float v = sb[i];
  if (!isfinite(v) || !(v >= thresh)) return false;
  for (int dy = -kNms; dy <= kNms; ++dy)
    for (int dx = -kNms; dx <= kNms; ++dx) {
      const float n = sb[i + (int64_t)dy * W + dx];
      if (isfinite(n) && n > v) return false;
    }
  return true;
}

__global__ void __launch_bounds__(256)
k_cand_count(int H, int W, const float* __restrict__ snr, const uint8_t* __restrict__ bad, float thresh,
             int* __restrict__ rowcnt) {
  const int b = blockIdx.y, y = blockIdx.x;
  const int64_t img = (int64_t)H * W;
  int c = 0;
  if (y >= kMargin && y < H - kMargin)
    for (int x = kMargin + threadIdx.x; x < W - kMargin; x += blockDim.x)
      c += is_candidate(snr + b * img, bad ? bad + b * img : nullptr, W, y, x, thresh);
  c = __reduce_add_sync(0xffffffffu, c);
  __shared__ int red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < 8; ++w) s += red[w];
    rowcnt[(int64_t)b * H + y] = s;
  }
}

// exclusive scan of the row counts of one CCD; count[b] = total
__global__ void __launch_bounds__(1024)
k_cand_scan(int H, const int* __restrict__ rowcnt, int* __restrict__ rowoff, int32_t* __restrict__ count) {
  __shared__ int part[1024];
  const int b = blockIdx.x, t = threadIdx.x;
  const int per = (H + 1023) / 1024;
  const int y0 = t * per;
  int s = 0;
  for (int k = 0; k < per; ++k)
    if (y0 + k < H) s += rowcnt[(int64_t)b * H + y0 + k];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;
  for (int k = 0; k < per; ++k)
    if (y0 + k < H) {
      rowoff[(int64_t)b * H + y0 + k] = run;
      run += rowcnt[(int64_t)b * H + y0 + k];
    }
  if (t == 1023) count[b] = part[1023];
}

__global__ void __launch_bounds__(256)
k_cand_write(int H, int W, const float* __restrict__ snr, const uint8_t* __restrict__ bad, float thresh,
             const int* __restrict__ rowcnt, const int* __restrict__ rowoff, int max_cand, int32_t* __restrict__ xy,
             float* __restrict__ osnr) {
  const int b = blockIdx.y, y = blockIdx.x;
  if (rowcnt[(int64_t)b * H + y] == 0) return;
  const int64_t img = (int64_t)H * W;
  const float* sb = snr + b * img;
  const uint8_t* bb = bad ? bad + b * img : nullptr;
  __shared__ int wtot[8];
  int base = rowoff[(int64_t)b * H + y];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int x0 = kMargin; x0 < W - kMargin; x0 += blockDim.x) {
    const int x = x0 + threadIdx.x;
    const bool c = x < W - kMargin && is_candidate(sb, bb, W, y, x, thresh);
    const unsigned m = __ballot_sync(0xffffffffu, c);
    if (lane == 0) wtot[warp] = __popc(m);
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < 8; ++w) {
      before += w < warp ? wtot[w] : 0;
      total += wtot[w];
    }
    if (c) {
      const int idx = base + before + __popc(m & ((1u << lane) - 1u));
      if (idx < max_cand) {
        xy[((int64_t)b * max_cand + idx) * 2 + 0] = x;
        xy[((int64_t)b * max_cand + idx) * 2 + 1] = y;
        osnr[(int64_t)b * max_cand + idx] = sb[(int64_t)y * W + x];
      }
    }
    base += total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
k_stamps(int H, int W, const float* __restrict__ S, const float* __restrict__ R, const float* __restrict__ D,
         const int32_t* __restrict__ count, const int32_t* __restrict__ xy, int max_cand, float* __restrict__ stamps) {
  const int b = blockIdx.y, i = blockIdx.x;
  const int n = min(count[b], max_cand);
  if (i >= n) return;
  const int x = xy[((int64_t)b * max_cand + i) * 2], y = xy[((int64_t)b * max_cand + i) * 2 + 1];
  const int64_t img = (int64_t)H * W;
  const int side = 2 * kHalf + 1, pix = side * side;
  float* out = stamps + ((int64_t)b * max_cand + i) * 3 * pix;
  for (int e = threadIdx.x; e < 3 * pix; e += blockDim.x) {
    const int ch = e / pix, p = e % pix;
    const int yy = y - kHalf + p / side, xx = x - kHalf + p % side;
    const float* src = ch == 0 ? S : (ch == 1 ? R : D);
    const float v = src[b * img + (int64_t)yy * W + xx];
    out[e] = isfinite(v) ? v : 0.f;
  }
}

// one thread per stamp; FP64 moments of the difference channel
__global__ void k_shape_cuts(const float* __restrict__ stamps, const float* __restrict__ snr, int64_t n,
                             double psf_fwhm, double snr_min, int32_t* __restrict__ pass) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int side = 2 * kHalf + 1;
  const float* d = stamps + (i * 3 + 2) * side * side;
  const int c = kHalf;
  double tot = 0.0, sx = 0.0, sy = 0.0;
  for (int yy = -4; yy <= 4; ++yy)
    for (int xx = -4; xx <= 4; ++xx) {
      const double p = fmax((double)d[(c + yy) * side + c + xx], 0.0);
      tot += p;
      sx += p * xx;
      sy += p * yy;
    }
  if (!((double)snr[i] >= snr_min) || !(tot > 0.0)) {
    pass[i] = 0;
    return;
  }
  const double mx = sx / tot, my = sy / tot;
  double sxx = 0.0, syy = 0.0, sxy = 0.0;
  for (int yy = -4; yy <= 4; ++yy)
    for (int xx = -4; xx <= 4; ++xx) {
      const double p = fmax((double)d[(c + yy) * side + c + xx], 0.0);
      sxx += p * (xx - mx) * (xx - mx);
      syy += p * (yy - my) * (yy - my);
      sxy += p * (xx - mx) * (yy - my);
    }
  sxx /= tot;
  syy /= tot;
  sxy /= tot;
  const double tr = sxx + syy, det = sxx * syy - sxy * sxy;
  const double disc = sqrt(fmax(tr * tr / 4.0 - det, 0.0));
  const double l1 = tr / 2.0 + disc, l2 = fmax(tr / 2.0 - disc, 1e-12);
  const double fwhm = 2.0 * sqrt(2.0 * log(2.0)) * sqrt(fmax(0.5 * (l1 + l2), 0.0));
  double neg = 0.0, absum = 0.0;
  for (int yy = -3; yy <= 3; ++yy)
    for (int xx = -3; xx <= 3; ++xx) {
      const double v = (double)d[(c + yy) * side + c + xx];
      neg += fabs(fmin(v, 0.0));
      absum += fabs(v);
    }
  const double neg_frac = neg / fmax(absum, 1e-12);
  const double ratio = sqrt(l1 / l2);
  pass[i] = (0.5 * psf_fwhm <= fwhm && fwhm <= 2.0 * psf_fwhm && neg_frac < 0.3 && ratio < 2.5) ? 1 : 0;
}

// The same cuts with the size and axis ratio from Gaussian-weighted adaptive
// moments of the difference channel over the central 15 x 15: from a round
// weight of the PSF's width at the centre, 40 times w = exp(-(r - mu)^T M^-1
// (r - mu) / 2), mu = sum w I r / sum w I, M = 2 sum w I (r - mu)(r - mu)^T /
// sum w I (a Gaussian source of covariance C is the fixed point M = C); a
// candidate whose weighted flux is not positive, whose M is not positive
// definite, whose centroid moves more than 3 px or whose M grows past
// 25 px^2 fails.  One thread per stamp, FP64.
constexpr int kAmHalf = 7, kAmIters = 40;

__global__ void k_shape_cuts_adaptive(const float* __restrict__ stamps, const float* __restrict__ snr, int64_t n,
                                      double psf_fwhm, double snr_min, int32_t* __restrict__ pass) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int side = 2 * kHalf + 1;
  const float* d = stamps + (i * 3 + 2) * side * side;
  const int c = kHalf;
  const double fw2s = 2.0 * sqrt(2.0 * log(2.0));
  const double s0w = psf_fwhm / fw2s;
  double mxx = s0w * s0w, myy = s0w * s0w, mxy = 0.0, mx = 0.0, my = 0.0;
  bool ok = (double)snr[i] >= snr_min;
  for (int it = 0; ok && it < kAmIters; ++it) {
    const double det = mxx * myy - mxy * mxy;
    if (!(det > 0.0 && mxx > 0.0 && myy > 0.0)) { ok = false; break; }
    const double ia = myy / det, ib = -mxy / det, ic = mxx / det;   // M^-1 = [[ia, ib], [ib, ic]]
    double s0 = 0.0, sx = 0.0, sy = 0.0, sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (int yy = -kAmHalf; yy <= kAmHalf; ++yy)
      for (int xx = -kAmHalf; xx <= kAmHalf; ++xx) {
        const double dx = xx - mx, dy = yy - my;
        const double wv = exp(-0.5 * (ia * dx * dx + 2.0 * ib * dx * dy + ic * dy * dy)) *
                          (double)d[(c + yy) * side + c + xx];
        s0 += wv;
        sx += wv * xx;
        sy += wv * yy;
        sxx += wv * xx * xx;
        syy += wv * yy * yy;
        sxy += wv * xx * yy;
      }
    if (!(s0 > 0.0)) { ok = false; break; }
    mx = sx / s0;
    my = sy / s0;
    // central moments about the new centroid from the raw sums
    mxx = 2.0 * (sxx / s0 - mx * mx);
    myy = 2.0 * (syy / s0 - my * my);
    mxy = 2.0 * (sxy / s0 - mx * my);
    if (fabs(mx) > 3.0 || fabs(my) > 3.0 || mxx > 25.0 || myy > 25.0) ok = false;
  }
  if (ok && !(mxx * myy - mxy * mxy > 0.0 && mxx > 0.0 && myy > 0.0)) ok = false;
  if (!ok) {
    pass[i] = 0;
    return;
  }
  const double tr = mxx + myy, det = mxx * myy - mxy * mxy;
  const double disc = sqrt(fmax(tr * tr / 4.0 - det, 0.0));
  const double l1 = tr / 2.0 + disc, l2 = fmax(tr / 2.0 - disc, 1e-12);
  const double fwhm = fw2s * sqrt(0.5 * (l1 + l2));
  double neg = 0.0, absum = 0.0;
  for (int yy = -3; yy <= 3; ++yy)
    for (int xx = -3; xx <= 3; ++xx) {
      const double v = (double)d[(c + yy) * side + c + xx];
      neg += fabs(fmin(v, 0.0));
      absum += fabs(v);
    }
  const double neg_frac = neg / fmax(absum, 1e-12);
  const double ratio = sqrt(l1 / l2);
  pass[i] = (0.5 * psf_fwhm <= fwhm && fwhm <= 2.0 * psf_fwhm && neg_frac < 0.3 && ratio < 2.5) ? 1 : 0;
}

sfft_status_t fail(cudaError_t e, const char* where) {
  sfft::set_last_error((std::string(where) + ": " + cudaGetErrorString(e)).c_str());
  return SFFT_ERR_CUDA;
}

}  // namespace

extern "C" size_t rb_detect_workspace_bytes(int32_t H, int32_t W, int32_t batch, int32_t max_cand) {
  (void)max_cand;
  if (H < 1 || W < 1 || batch < 1) return 0;
  return DetectLayout(H, W, batch).total;
}

extern "C" sfft_status_t rb_detect(int32_t H, int32_t W, int32_t batch, const float* D, const float* S,
                                   const float* R, const uint8_t* bad, float psf_sigma, float thresh,
                                   int32_t guard, int32_t max_cand, int32_t* xy, float* snr, int32_t* count, float* stamps, void* ws,
                                   void* stream) {
  if (H < 2 * kHalf + 1 || W < 2 * kHalf + 1 || batch < 1 || max_cand < 0 || !D || !S || !R || !count || !ws ||
      (max_cand > 0 && (!xy || !snr || !stamps)) || !(psf_sigma > 0.f) || !(psf_sigma <= 5.f) || guard < 0 ||
      guard > kMargin ||
      (reinterpret_cast<uintptr_t>(ws) & 255))
    return SFFT_ERR_ARG;
  if (batch > 65535 || sizeof(float) * (W + 2 * kMaxR) > 48 * 1024) return SFFT_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const DetectLayout L(H, W, batch);
  char* base = static_cast<char*>(ws);
  float* snr_map = reinterpret_cast<float*>(base + L.snr);
  float* tmp = reinterpret_cast<float*>(base + L.tmp);
  double* part = reinterpret_cast<double*>(base + L.part);
  int* rowcnt = reinterpret_cast<int*>(base + L.rowcnt);
  int* rowoff = reinterpret_cast<int*>(base + L.rowoff);

  Taps taps{};
  taps.r = (int)ceil(3.0 * (double)psf_sigma);
  for (int k = 0; k <= 2 * taps.r; ++k) {
    const double t = k - taps.r;
    taps.g[k] = (float)exp(-t * t / (2.0 * (double)psf_sigma * (double)psf_sigma));
  }
  for (int p = 0; p < kStatPasses; ++p) k_clip_pass<<<dim3(kStatBlocks, batch), 256, 0, s>>>(H, W, D, bad, part, p);
  const size_t row_smem = sizeof(float) * (W + 2 * taps.r);
  k_filter_rows<<<dim3(std::min(H, 1024), batch), 256, row_smem, s>>>(H, W, D, bad, taps, tmp);
  k_filter_cols<<<dim3((W + 31) / 32, (H + kColTile - 1) / kColTile, batch), 256, 0, s>>>(H, W, tmp, taps, part,
                                                                                             snr_map);
  const uint8_t* cbad = bad;   // the mask the candidate test reads
  if (bad && guard > 0) {
    uint8_t* rows = reinterpret_cast<uint8_t*>(base + L.tmp);    // the row-filtered image is consumed by now
    uint8_t* gm = reinterpret_cast<uint8_t*>(base + L.guard);
    const int gx = (int)std::min<int64_t>(((int64_t)H * W + 255) / 256, 2048);
    k_dilate_rows<<<dim3(gx, batch), 256, 0, s>>>(H, W, bad, guard, rows);
    k_dilate_cols<<<dim3(gx, batch), 256, 0, s>>>(H, W, rows, guard, gm);
    cbad = gm;
  }
  k_cand_count<<<dim3(H, batch), 256, 0, s>>>(H, W, snr_map, cbad, thresh, rowcnt);
  k_cand_scan<<<batch, 1024, 0, s>>>(H, rowcnt, rowoff, count);
  if (max_cand > 0) {
    k_cand_write<<<dim3(H, batch), 256, 0, s>>>(H, W, snr_map, cbad, thresh, rowcnt, rowoff, max_cand, xy, snr);
    k_stamps<<<dim3(max_cand, batch), 256, 0, s>>>(H, W, S, R, D, count, xy, max_cand, stamps);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rb_detect");
}

extern "C" sfft_status_t rb_shape_cuts(const float* stamps, const float* snr, int64_t n, float psf_fwhm,
                                       float snr_min, int32_t* pass, void* stream) {
  if (n < 0 || (n > 0 && (!stamps || !snr || !pass)) || !(psf_fwhm > 0.f)) return SFFT_ERR_ARG;
  if (n == 0) return SFFT_OK;
  k_shape_cuts<<<(unsigned)((n + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(stamps, snr, n, psf_fwhm,
                                                                                             snr_min, pass);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rb_shape_cuts");
}

extern "C" sfft_status_t rb_shape_cuts_adaptive(const float* stamps, const float* snr, int64_t n, float psf_fwhm,
                                                float snr_min, int32_t* pass, void* stream) {
  if (n < 0 || (n > 0 && (!stamps || !snr || !pass)) || !(psf_fwhm > 0.f)) return SFFT_ERR_ARG;
  if (n == 0) return SFFT_OK;
  k_shape_cuts_adaptive<<<(unsigned)((n + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
      stamps, snr, n, psf_fwhm, snr_min, pass);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rb_shape_cuts_adaptive");
}
