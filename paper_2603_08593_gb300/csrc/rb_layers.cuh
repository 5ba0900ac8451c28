// Layers shared by the stamp classifiers (rb_cnn.cu: the small network;
// rb_ri.cu: the rotation-invariant residual network): implicit-GEMM
// launchers, the robust per-channel normalisation, ReLU / max-pool and their
// backward passes, the dense head, bias-gradient column sums, Adam.
#pragma once
#include <math.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "rb_gemm.cuh"

namespace {

using bf16 = __nv_bfloat16;
constexpr int S31 = 31, PIX1 = 961, PIX2 = 225, PIX3 = 49, PIX4 = 9;
constexpr int C1 = 32, C2 = 64, C3 = 64, F4 = 128;
constexpr int K1 = 32, K2 = 9 * C1, K3 = 9 * C2, K4 = PIX4 * C3;   // GEMM K (conv1 padded)

// ---------------------------------------------------------------- GEMM launchers
constexpr int kMaxSplits = 64;

// out[e] = sum over z of part[z mn + e], one warp per element: lane l adds
// slices l, l + 32, ... in order, then a fixed xor tree (deterministic)
__global__ void __launch_bounds__(256)
k_sum_splits(const float* __restrict__ part, int splits, int64_t mn, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); e < mn; e += nw) {
    float s = 0.f;
    for (int z = lane; z < splits; z += 32) s += part[z * mn + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[e] = s;
  }
}

inline cudaError_t sum_splits(cudaStream_t s, const float* part, int splits, int64_t mn, float* out) {
  k_sum_splits<<<(int)std::min<int64_t>((mn + 7) / 8, 4096), 256, 0, s>>>(part, splits, mn, out);
  return cudaGetLastError();
}

// C = A B (+ bias): A K-major (rows = M), B outer-major (rows = K) or K-major (rows = N)
template <class LA, class LB, bool B_KM>
cudaError_t igemm(cudaStream_t s, int M, int N, int K, const LA& la, const LB& lb, float* C, int ldc,
                  const float* bias) {
  dim3 grid((N + rbg::BN - 1) / rbg::BN, (M + rbg::BM - 1) / rbg::BM, 1);
  rbg::k_igemm<LA, LB, true, B_KM, false><<<grid, 256, 0, s>>>(M, N, K, K, la, lb, C, ldc, 0, bias);
  return cudaGetLastError();
}

// Weight gradient G[n][m] (ldc = M) = sum_k A[k][m] B[k][n] over a long k
// (pixels or stamps): both operands outer-major, split over k into fixed
// slices of `part` (kMaxSplits * K4 * F4 floats, so up to that many / (M N)
// slices) summed in a fixed order.  About four CTAs per SM: the small
// products (conv1: M = N = 32 over 961 pixels a stamp) get many slices.
template <class LA, class LB>
cudaError_t igemm_wgrad(cudaStream_t s, int M, int N, int K, const LA& la, const LB& lb, float* G, float* part) {
  const int tiles = ((N + rbg::BN - 1) / rbg::BN) * ((M + rbg::BM - 1) / rbg::BM);
  const int64_t cap = (int64_t)kMaxSplits * K4 * F4 / ((int64_t)M * N);
  int splits = (int)std::min<int64_t>({(int64_t)(K + 255) / 256, cap, (int64_t)std::max(1, 4 * 152 / tiles)});
  splits = std::max(splits, 1);
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + rbg::BK - 1) / rbg::BK * rbg::BK;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid((N + rbg::BN - 1) / rbg::BN, (M + rbg::BM - 1) / rbg::BM, splits);
  const int64_t mn = (int64_t)M * N;
  float* dst = splits == 1 ? G : part;
  rbg::k_igemm<LA, LB, false, false, true><<<grid, 256, 0, s>>>(M, N, K, kchunk, la, lb, dst, M, mn, nullptr);
  if (splits > 1)
    sum_splits(s, part, splits, mn, G);
  return cudaGetLastError();
}

// B operand of the input gradient: row = ci, k = (tap, co) -> W[(tap * cin + ci)][co .. co + 7]
struct ConvW {
  const bf16* w;
  int cin, cout;
  __device__ __forceinline__ uint4 row8(int ci, int k) const {
    if (ci >= cin || k >= 9 * cout) return rbg::zero4();
    const int tap = k / cout, co = k - tap * cout;
    return *reinterpret_cast<const uint4*>(w + ((int64_t)tap * cin + ci) * cout + co);
  }
};

// ---------------------------------------------------------------- elementwise kernels
// Robust normalisation: x -> clip((x - median) / (1.4826 MAD), +-64) per
// stamp and channel (scale 1 when the MAD is 0), output NHWC BF16 with
// `stride` values per stamp (961 x 3 = 2883, or 2888 so that every stamp
// starts on a 16-byte boundary; the pad is zero).  One block of three warps
// per stamp, one warp per channel.  The median and the MAD are exact order
// statistics (the 481st smallest of 961 values) found without a full sort:
// each lane sorts its 31 values (padded with +inf to 32) in registers, and a
// bisection over the order-preserving integer image of the FP32 values
// counts, per probe, the values <= the probe in every lane's sorted column
// (a 5-step search in shared memory) until the smallest value with at least
// 481 values <= it is found.  The absolute deviations of a sorted column
// fall and then rise, so one bitonic merge sorts them for the second search.
__device__ __forceinline__ void sort32(float (&v)[32]) {
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const float a = v[i], b = v[l];
          v[i] = up ? fminf(a, b) : fmaxf(a, b);
          v[l] = up ? fmaxf(a, b) : fminf(a, b);
        }
      }
}

// ascending sort of a sequence that first falls and then rises (bitonic)
__device__ __forceinline__ void merge32(float (&v)[32]) {
#pragma unroll
  for (int j = 16; j > 0; j >>= 1)
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int l = i ^ j;
      if (l > i) {
        const float a = v[i], b = v[l];
        v[i] = fminf(a, b);
        v[l] = fmaxf(a, b);
      }
    }
}

__device__ __forceinline__ uint32_t order_key(float x) {
  const uint32_t b = __float_as_uint(x);
  return b ^ ((b >> 31) ? 0xffffffffu : 0x80000000u);
}
__device__ __forceinline__ float key_value(uint32_t k) {
  return __uint_as_float(k ^ ((k >> 31) ? 0x80000000u : 0xffffffffu));
}

// The (rank + 1)-th smallest of the warp's finite values: v is the lane's
// sorted column (finite entries first, nfin of them, then +inf), col the
// lane's column in shared memory ([32][32], entry r of lane l at r * 32 + l).
__device__ __forceinline__ float warp_select(const float (&v)[32], int nfin, float* col, int rank) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < 32; ++r) col[r * 32 + lane] = v[r];
  __syncwarp();
  float vmax = v[0];
#pragma unroll
  for (int r = 1; r < 32; ++r) vmax = r < nfin ? v[r] : vmax;
  uint32_t lo = __reduce_min_sync(0xffffffffu, order_key(v[0]));
  uint32_t hi = __reduce_max_sync(0xffffffffu, order_key(vmax));
  while (lo < hi) {   // smallest key with more than `rank` values <= it
    const uint32_t mid = lo + ((hi - lo) >> 1);
    const float p = key_value(mid);
    int pos = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) pos += col[(pos + step - 1) * 32 + lane] <= p ? step : 0;
    const int c = (int)__reduce_add_sync(0xffffffffu, (unsigned)pos);
    if (c > rank) hi = mid;
    else lo = mid + 1;
  }
  __syncwarp();
  return key_value(hi);
}

__global__ void __launch_bounds__(96)
k_normalise(const float* __restrict__ stamps, int n, bf16* __restrict__ xn, int stride) {
  __shared__ float cols[3][32 * 32];
  __shared__ __align__(16) bf16 stage[2888];
  const int st = blockIdx.x, ch = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (st >= n) return;
  const float* src = stamps + ((int64_t)st * 3 + ch) * PIX1;
  float v[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int i = r * 32 + lane;
    v[r] = (r < 31 && i < PIX1) ? src[i] : INFINITY;
  }
  const int nfin = lane == 0 ? 31 : 30;   // 961 = 30 x 32 + 1
  sort32(v);
  const float med = warp_select(v, nfin, cols[ch], 480);
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = fabsf(v[r] - med);   // +inf stays +inf, at the end
  merge32(v);
  const float sc = 1.4826f * warp_select(v, nfin, cols[ch], 480);
  const float inv = 1.f / (sc > 0.f ? sc : 1.f);
  for (int i = lane; i < PIX1; i += 32) {
    const float x = fminf(fmaxf((src[i] - med) * inv, -64.f), 64.f);
    stage[i * 3 + ch] = __float2bfloat16(x);
  }
  if (threadIdx.x < stride - 3 * PIX1) stage[3 * PIX1 + threadIdx.x] = __float2bfloat16(0.f);
  __syncthreads();
  bf16* dst = xn + (int64_t)st * stride;
  if (stride % 8 == 0) {
    for (int i = threadIdx.x; i < stride / 8; i += blockDim.x)
      reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(stage)[i];
  } else {
    for (int i = threadIdx.x; i < stride; i += blockDim.x) dst[i] = stage[i];
  }
}

// ReLU + 2 x 2 max-pool (floor): z [n][h][w][c] -> a (bf16) [n][h/2][w/2][c], idx (first max in (0,0),(0,1),(1,0),(1,1))
__global__ void k_relu_pool(const float* __restrict__ z, int n, int h, int w, int c, bf16* __restrict__ a,
                            uint8_t* __restrict__ idx) {
  const int ho = h / 2, wo = w / 2;
  const int64_t total = (int64_t)n * ho * wo * c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int ci = (int)(e % c);
    const int64_t p = e / c;
    const int xo = (int)(p % wo), yo = (int)((p / wo) % ho), nn = (int)(p / ((int64_t)wo * ho));
    float best = -INFINITY;
    int bi = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int yy = 2 * yo + (q >> 1), xx = 2 * xo + (q & 1);
      const float v = fmaxf(z[(((int64_t)nn * h + yy) * w + xx) * c + ci], 0.f);
      if (v > best) { best = v; bi = q; }
    }
    a[e] = __float2bfloat16(best);
    if (idx) idx[e] = (uint8_t)bi;
  }
}

// pool + ReLU backward: dz[n][h][w][c] = (position == argmax) * da * (z > 0); bf16 output
__global__ void k_pool_relu_back(const float* __restrict__ da, const uint8_t* __restrict__ idx,
                                 const float* __restrict__ z, int n, int h, int w, int c, bf16* __restrict__ dz) {
  // one thread per (pixel, 8 channels): 32-byte loads of z and da, 8 bytes of
  // indices, a 16-byte store of dz (c is a multiple of 8)
  const int ho = h / 2, wo = w / 2, c8 = c / 8;
  const int64_t total = (int64_t)n * h * w * c8;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % c8);
    const int64_t p = t / c8;
    const int pix = (int)(p % ((int64_t)h * w)), nn = (int)(p / ((int64_t)h * w));
    const int yy = pix / w, xx = pix - yy * w, yo = yy >> 1, xo = xx >> 1;
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (yo < ho && xo < wo) {
      const int64_t e = p * c + 8 * q;
      const float4 z0 = *reinterpret_cast<const float4*>(z + e), z1 = *reinterpret_cast<const float4*>(z + e + 4);
      const int64_t pe = (((int64_t)nn * ho + yo) * wo + xo) * c + 8 * q;
      const uint2 ix = *reinterpret_cast<const uint2*>(idx + pe);
      const float4 d0 = *reinterpret_cast<const float4*>(da + pe), d1 = *reinterpret_cast<const float4*>(da + pe + 4);
      const float zz[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
      const float dd[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
      const uint32_t pos = (uint32_t)(((yy & 1) << 1) | (xx & 1));
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint32_t ib = ((i < 4 ? ix.x : ix.y) >> (8 * (i & 3))) & 0xffu;
        v[i] = (zz[i] > 0.f && ib == pos) ? dd[i] : 0.f;
      }
    }
    __align__(16) bf16 o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) o[i] = __float2bfloat16(v[i]);
    *reinterpret_cast<uint4*>(dz + p * c + 8 * q) = *reinterpret_cast<const uint4*>(o);
  }
}

// dense layer: z5 = relu(z4) . w5 + b5 (FP32, one warp per sample); NaN
// logits when `err` (optional) reports a failed step earlier in the forward
__global__ void k_fc2(const float* __restrict__ z4, const float* __restrict__ w5, const float* __restrict__ b5,
                      int n, float* __restrict__ logit, const int* __restrict__ err = nullptr) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  float s = 0.f;
  for (int i = lane; i < F4; i += 32) s += fmaxf(z4[(int64_t)warp * F4 + i], 0.f) * w5[i];
  s = sfft::warp_sum(s);
  if (lane == 0) logit[warp] = (err && *err) ? __int_as_float(0x7fc00000) : s + b5[0];
}

__global__ void k_sigmoid(const float* __restrict__ z, int64_t n, float* __restrict__ s) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s[e] = 1.f / (1.f + expf(-z[e]));
}

// BCE head: loss (mean), dz5 = (sigmoid - t) / n; then dW5, db5, dz4 = dz5 w5 (z4 > 0) (bf16)
__global__ void k_bce_head(const float* __restrict__ logit, const float* __restrict__ target, int n,
                           const float* __restrict__ z4, const float* __restrict__ w5, float* __restrict__ dz5,
                           bf16* __restrict__ dz4, float* __restrict__ loss_dev) {
  __shared__ float red[32];
  float l = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float z = logit[i], t = target[i];
    l += fmaxf(z, 0.f) - z * t + log1pf(expf(-fabsf(z)));
    dz5[i] = (1.f / (1.f + expf(-z)) - t) / (float)n;
  }
  l = sfft::warp_sum(l);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x < 32) {
    float s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    s = sfft::warp_sum(s);
    if (threadIdx.x == 0 && loss_dev) *loss_dev = s / (float)n;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)n * F4; e += blockDim.x) {
    const int i = (int)(e / F4), j = (int)(e % F4);
    dz4[e] = __float2bfloat16(z4[e] > 0.f ? dz5[i] * w5[j] : 0.f);
  }
}

// dw5[j] = sum_i dz5[i] relu(z4[i][j]), db5 = sum_i dz5[i]: one warp per j
// (lane l adds samples l, l + 32, ... in order, then a fixed xor tree); the
// warp of j = 0 also forms db5.  Launch F4 / 8 CTAs of 256 threads.
__global__ void __launch_bounds__(256)
k_fc2_grad(const float* __restrict__ dz5, const float* __restrict__ z4, int n, float* __restrict__ dw5,
           float* __restrict__ db5) {
  const int lane = threadIdx.x & 31, j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= F4) return;   // whole warps
  float s = 0.f, sb = 0.f;
  for (int i = lane; i < n; i += 32) {
    const float d = dz5[i];
    s += d * fmaxf(z4[(int64_t)i * F4 + j], 0.f);
    sb += d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  if (lane == 0) {
    dw5[j] = s;
    if (j == 0) db5[0] = sb;
  }
}

// column sums of a bf16 matrix [rows][cols] into FP32 (bias gradients), cols
// dividing 256: each CTA sums a band of rows with coalesced reads into
// part[blockIdx.x][cols]; the bands are then added in a fixed order.
__global__ void __launch_bounds__(256)
k_colsum_part(const bf16* __restrict__ x, int64_t rows, int cols, int64_t band, float* __restrict__ part) {
  __shared__ float red[256];
  const int c = threadIdx.x % cols, rp = threadIdx.x / cols, nrp = blockDim.x / cols;
  const int64_t r0 = blockIdx.x * band, r1 = min(rows, r0 + band);
  float s = 0.f;
  for (int64_t r = r0 + rp; r < r1; r += nrp) s += __bfloat162float(x[r * cols + c]);
  red[threadIdx.x] = s;
  __syncthreads();
  if (rp == 0) {
    for (int q = 1; q < nrp; ++q) s += red[q * cols + c];
    part[(int64_t)blockIdx.x * cols + c] = s;
  }
}

cudaError_t colsum(cudaStream_t st, const bf16* x, int64_t rows, int cols, float* part, float* out) {
  const int nb = (int)std::min<int64_t>(512, (rows + 255) / 256);
  const int64_t band = (rows + nb - 1) / nb;
  k_colsum_part<<<nb, 256, 0, st>>>(x, rows, cols, band, part);
  sum_splits(st, part, nb, cols, out);
  return cudaGetLastError();
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float c1, float c2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float ge = g[e];
    const float me = 0.9f * m[e] + 0.1f * ge;
    const float ve = 0.999f * v[e] + 0.001f * ge * ge;
    m[e] = me;
    v[e] = ve;
    p[e] -= lr * (me / c1) / (sqrtf(ve / c2) + 1e-8f);
  }
}

__global__ void k_to_bf16(const float* __restrict__ x, int64_t n, bf16* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = __float2bfloat16(x[e]);
}

int grid1(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

// splitmix64 -> uniform in [0, 1)
double hash_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed * 0x9E3779B97F4A7C15ull + i + 0x632BE59BD9B4E019ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace
