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

__global__ void k_sum_splits(const float* __restrict__ part, int splits, int64_t mn, float* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < mn; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[z * mn + e];
    out[e] = s;
  }
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
// slices of `part` (kMaxSplits * M * N floats) summed in a fixed order.
template <class LA, class LB>
cudaError_t igemm_wgrad(cudaStream_t s, int M, int N, int K, const LA& la, const LB& lb, float* G, float* part) {
  const int tiles = ((N + rbg::BN - 1) / rbg::BN) * ((M + rbg::BM - 1) / rbg::BM);
  int splits = std::min({(K + 1023) / 1024, kMaxSplits, std::max(1, 2 * 152 / tiles)});
  splits = std::max(splits, 1);
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + rbg::BK - 1) / rbg::BK * rbg::BK;
  splits = (K + kchunk - 1) / kchunk;
  dim3 grid((N + rbg::BN - 1) / rbg::BN, (M + rbg::BM - 1) / rbg::BM, splits);
  const int64_t mn = (int64_t)M * N;
  float* dst = splits == 1 ? G : part;
  rbg::k_igemm<LA, LB, false, false, true><<<grid, 256, 0, s>>>(M, N, K, kchunk, la, lb, dst, M, mn, nullptr);
  if (splits > 1)
    k_sum_splits<<<(int)std::min<int64_t>((mn + 255) / 256, 1024), 256, 0, s>>>(part, splits, mn, G);
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
// Robust normalisation of one channel of one stamp per warp: the 961 values
// (padded with +inf to 1024) are sorted in registers by a bitonic network
// (position p = lane * 32 + r; partner positions in other lanes are reached by
// shuffles), the median is position 480; the absolute deviations are sorted
// the same way for the MAD.  x -> clip((x - median) / (1.4826 MAD), +-64),
// scale 1 when the MAD is 0.  Output NHWC BF16 [n][31][31][3].
__device__ __forceinline__ void warp_bitonic_1024(float (&v)[32], int lane) {
#pragma unroll
  for (int k = 2; k <= 1024; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int lj = j >> 5;
        const bool lower = (lane & lj) == 0;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const bool up = (((lane * 32 + r) & k) == 0);
          const float o = __shfl_xor_sync(0xffffffffu, v[r], lj);
          v[r] = (lower == up) ? fminf(v[r], o) : fmaxf(v[r], o);
        }
      } else {
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int rp = r ^ j;
          if (rp > r) {
            const bool up = (((lane * 32 + r) & k) == 0);
            const float x = v[r], y = v[rp];
            v[r] = up ? fminf(x, y) : fmaxf(x, y);
            v[rp] = up ? fmaxf(x, y) : fminf(x, y);
          }
        }
      }
    }
  }
}

__global__ void __launch_bounds__(256)
k_normalise(const float* __restrict__ stamps, int n, bf16* __restrict__ xn) {
  const int lane = threadIdx.x & 31;
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);   // (stamp, channel)
  if (item >= 3 * n) return;                                              // whole warps
  const int st = item / 3, ch = item - 3 * st;
  const float* src = stamps + ((int64_t)st * 3 + ch) * PIX1;
  float v[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int i = r * 32 + lane;
    v[r] = i < PIX1 ? src[i] : INFINITY;
  }
  warp_bitonic_1024(v, lane);
  const float med = __shfl_sync(0xffffffffu, v[0], 15);   // position 480
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int i = r * 32 + lane;
    v[r] = i < PIX1 ? fabsf(src[i] - med) : INFINITY;
  }
  warp_bitonic_1024(v, lane);
  const float sc = 1.4826f * __shfl_sync(0xffffffffu, v[0], 15);
  const float inv = 1.f / (sc > 0.f ? sc : 1.f);
  for (int i = lane; i < PIX1; i += 32) {
    const float x = fminf(fmaxf((src[i] - med) * inv, -64.f), 64.f);
    xn[((int64_t)st * PIX1 + i) * 3 + ch] = __float2bfloat16(x);
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
  const int ho = h / 2, wo = w / 2;
  const int64_t total = (int64_t)n * h * w * c;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int ci = (int)(e % c);
    const int64_t p = e / c;
    const int xx = (int)(p % w), yy = (int)((p / w) % h), nn = (int)(p / ((int64_t)w * h));
    float v = 0.f;
    const int yo = yy / 2, xo = xx / 2;
    if (yo < ho && xo < wo && z[e] > 0.f) {
      const int64_t pe = (((int64_t)nn * ho + yo) * wo + xo) * c + ci;
      if (idx[pe] == (uint8_t)(((yy & 1) << 1) | (xx & 1))) v = da[pe];
    }
    dz[e] = __float2bfloat16(v);
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

// dw5[j] = sum_i dz5[i] relu(z4[i][j]); db5 = sum dz5
__global__ void k_fc2_grad(const float* __restrict__ dz5, const float* __restrict__ z4, int n, float* __restrict__ dw5,
                           float* __restrict__ db5) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < F4) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += dz5[i] * fmaxf(z4[(int64_t)i * F4 + j], 0.f);
    dw5[j] = s;
  }
  if (j == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += dz5[i];
    db5[0] = s;
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
  k_sum_splits<<<1, 256, 0, st>>>(part, nb, cols, out);
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
