// Stamp real-bogus classifier: BF16 tensor-core training and inference.
//
// Activations are NHWC.  Every convolution is an implicit GEMM (rb_gemm.cuh:
// no im2col matrix is written) on mma.sync m16n8k16 BF16 with FP32
// accumulation: forward  Z[pixel][co] = sum_k x(pixel + tap)[ci] W[k][co];
// weight gradient  dW[k][co] = sum_pixel dZ[pixel][co] x(pixel + tap)[ci]
// (split over pixels, partial sums added in a fixed order); input gradient
// dX[pixel][ci] = sum_(tap, co) dZ(pixel - tap)[co] W[(tap, ci)][co].  Master
// weights, gradients and Adam moments are FP32 and stored in GEMM layout:
// conv weights as [(ky*3 + kx)*cin + ci][cout] (conv1 padded from K = 27 to
// 32 with zero rows), the 576 -> 128 layer as [(i*3 + j)*64 + c][128];
// rb_set/get_weights convert from/to the [cout][cin][ky][kx] and
// channel-major flatten order of the C ABI.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "plan.h"
#include "rb.h"
#include "rb_gemm.cuh"

namespace {

using bf16 = __nv_bfloat16;
constexpr int S31 = 31, PIX1 = 961, PIX2 = 225, PIX3 = 49, PIX4 = 9;
constexpr int C1 = 32, C2 = 64, C3 = 64, F4 = 128;
constexpr int K1 = 32, K2 = 9 * C1, K3 = 9 * C2, K4 = PIX4 * C3;   // GEMM K (conv1 padded)

// master parameter offsets (GEMM layout, floats)
constexpr int OW1 = 0, OB1 = OW1 + K1 * C1, OW2 = OB1 + C1, OB2 = OW2 + K2 * C2, OW3 = OB2 + C2,
              OB3 = OW3 + K3 * C3, OW4 = OB3 + C3, OB4 = OW4 + K4 * F4, OW5 = OB4 + F4, OB5 = OW5 + F4,
              NMASTER = OB5 + 1;

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

// dense layer: z5 = relu(z4) . w5 + b5 (FP32, one warp per sample)
__global__ void k_fc2(const float* __restrict__ z4, const float* __restrict__ w5, const float* __restrict__ b5,
                      int n, float* __restrict__ logit) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  float s = 0.f;
  for (int i = lane; i < F4; i += 32) s += fmaxf(z4[(int64_t)warp * F4 + i], 0.f) * w5[i];
  s = sfft::warp_sum(s);
  if (lane == 0) logit[warp] = s + b5[0];
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

// ---------------------------------------------------------------- layout conversion (host)
// C-ABI order (oracle layout) <-> GEMM-layout master vector
void abi_to_master(const float* a, std::vector<float>& m) {
  m.assign(NMASTER, 0.f);
  const float* w1 = a;                      // [32][3][3][3]
  const float* b1 = w1 + 32 * 27;
  const float* w2 = b1 + 32;                // [64][32][3][3]
  const float* b2 = w2 + 64 * 288;
  const float* w3 = b2 + 64;                // [64][64][3][3]
  const float* b3 = w3 + 64 * 576;
  const float* w4 = b3 + 64;                // [128][576] (c*9 + i*3 + j)
  const float* b4 = w4 + 128 * 576;
  const float* w5 = b4 + 128;
  const float* b5 = w5 + 128;
  auto conv = [&](const float* w, int cin, int cout, int off) {
    for (int o = 0; o < cout; ++o)
      for (int ci = 0; ci < cin; ++ci)
        for (int ky = 0; ky < 3; ++ky)
          for (int kx = 0; kx < 3; ++kx)
            m[off + ((ky * 3 + kx) * cin + ci) * cout + o] = w[((o * cin + ci) * 3 + ky) * 3 + kx];
  };
  conv(w1, 3, C1, OW1);
  conv(w2, C1, C2, OW2);
  conv(w3, C2, C3, OW3);
  for (int i = 0; i < C1; ++i) m[OB1 + i] = b1[i];
  for (int i = 0; i < C2; ++i) m[OB2 + i] = b2[i];
  for (int i = 0; i < C3; ++i) m[OB3 + i] = b3[i];
  for (int o = 0; o < F4; ++o)
    for (int c = 0; c < C3; ++c)
      for (int p = 0; p < PIX4; ++p) m[OW4 + (p * C3 + c) * F4 + o] = w4[o * K4 + c * PIX4 + p];
  for (int i = 0; i < F4; ++i) m[OB4 + i] = b4[i];
  for (int i = 0; i < F4; ++i) m[OW5 + i] = w5[i];
  m[OB5] = b5[0];
}

void master_to_abi(const float* m, float* a) {
  float* w1 = a;
  float* b1 = w1 + 32 * 27;
  float* w2 = b1 + 32;
  float* b2 = w2 + 64 * 288;
  float* w3 = b2 + 64;
  float* b3 = w3 + 64 * 576;
  float* w4 = b3 + 64;
  float* b4 = w4 + 128 * 576;
  float* w5 = b4 + 128;
  float* b5 = w5 + 128;
  auto conv = [&](float* w, int cin, int cout, int off) {
    for (int o = 0; o < cout; ++o)
      for (int ci = 0; ci < cin; ++ci)
        for (int ky = 0; ky < 3; ++ky)
          for (int kx = 0; kx < 3; ++kx)
            w[((o * cin + ci) * 3 + ky) * 3 + kx] = m[off + ((ky * 3 + kx) * cin + ci) * cout + o];
  };
  conv(w1, 3, C1, OW1);
  conv(w2, C1, C2, OW2);
  conv(w3, C2, C3, OW3);
  for (int i = 0; i < C1; ++i) b1[i] = m[OB1 + i];
  for (int i = 0; i < C2; ++i) b2[i] = m[OB2 + i];
  for (int i = 0; i < C3; ++i) b3[i] = m[OB3 + i];
  for (int o = 0; o < F4; ++o)
    for (int c = 0; c < C3; ++c)
      for (int p = 0; p < PIX4; ++p) w4[o * K4 + c * PIX4 + p] = m[OW4 + (p * C3 + c) * F4 + o];
  for (int i = 0; i < F4; ++i) b4[i] = m[OB4 + i];
  for (int i = 0; i < F4; ++i) w5[i] = m[OW5 + i];
  b5[0] = m[OB5];
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

struct rb_model_s {
  int max_batch = 0;
  int64_t step = 0;
  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  bf16* wbf = nullptr;                         // bf16 copy of the master vector
  // activations / scratch for max_batch stamps
  bf16 *xn = nullptr, *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *dzb = nullptr, *dz4 = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *z3 = nullptr, *z4 = nullptr, *logit = nullptr, *dz5 = nullptr,
        *da = nullptr, *part = nullptr;
  uint8_t *i1 = nullptr, *i2 = nullptr, *i3 = nullptr;
};

namespace {

void free_model(rb_model_s* m) {
  void* ptrs[] = {m->params, m->grads, m->adam_m, m->adam_v, m->wbf, m->xn,  m->a1,   m->a2,   m->a3,
                  m->dzb,    m->dz4,   m->z1,     m->z2,     m->z3,  m->z4, m->logit, m->dz5,  m->da,
                  m->part,   m->i1,    m->i2,     m->i3};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

template <typename T>
bool alloc(T** p, size_t n) {
  return cudaMalloc((void**)p, sizeof(T) * (n > 0 ? n : 1)) == cudaSuccess;
}

// forward for n <= max_batch normalised stamps in m->xn; logits to m->logit
cudaError_t forward(rb_model_s* m, int n, cudaStream_t s, bool keep_idx) {
  using rbg::ConvRows;
  using rbg::Conv1Rows;
  using rbg::Dense;
  const bf16* W = m->wbf;
  const float* P = m->params;
  cudaError_t e;
  // conv1 (3 -> 32): implicit GEMM over the 27 (padded 32) taps x channels
  if ((e = igemm<Conv1Rows, Dense, false>(s, n * PIX1, C1, K1, Conv1Rows{m->xn, n, S31, S31},
                                          Dense{W + OW1, K1, C1, C1}, m->z1, C1, P + OB1)))
    return e;
  k_relu_pool<<<grid1((int64_t)n * PIX2 * C1), 256, 0, s>>>(m->z1, n, S31, S31, C1, m->a1, keep_idx ? m->i1 : nullptr);
  // conv2 (32 -> 64)
  if ((e = igemm<ConvRows, Dense, false>(s, n * PIX2, C2, K2, ConvRows{m->a1, n, 15, 15, C1, 1},
                                         Dense{W + OW2, K2, C2, C2}, m->z2, C2, P + OB2)))
    return e;
  k_relu_pool<<<grid1((int64_t)n * PIX3 * C2), 256, 0, s>>>(m->z2, n, 15, 15, C2, m->a2, keep_idx ? m->i2 : nullptr);
  // conv3 (64 -> 64)
  if ((e = igemm<ConvRows, Dense, false>(s, n * PIX3, C3, K3, ConvRows{m->a2, n, 7, 7, C2, 1},
                                         Dense{W + OW3, K3, C3, C3}, m->z3, C3, P + OB3)))
    return e;
  k_relu_pool<<<grid1((int64_t)n * PIX4 * C3), 256, 0, s>>>(m->z3, n, 7, 7, C3, m->a3, keep_idx ? m->i3 : nullptr);
  // fc1 (NHWC flatten of a3 matches the W4 rows) and fc2
  if ((e = igemm<Dense, Dense, false>(s, n, F4, K4, Dense{m->a3, n, K4, K4}, Dense{W + OW4, K4, F4, F4}, m->z4, F4,
                                      P + OB4)))
    return e;
  k_fc2<<<(n * 32 + 255) / 256, 256, 0, s>>>(m->z4, P + OW5, P + OB5, n, m->logit);
  return cudaGetLastError();
}

cudaError_t backward(rb_model_s* m, int n, const float* labels, float* loss_dev, cudaStream_t s) {
  using rbg::ConvRows;
  using rbg::Conv1Rows;
  using rbg::Dense;
  const bf16* W = m->wbf;
  float* G = m->grads;
  cudaError_t e;
  cudaMemsetAsync(G, 0, sizeof(float) * NMASTER, s);
  k_bce_head<<<1, 1024, 0, s>>>(m->logit, labels, n, m->z4, m->params + OW5, m->dz5, m->dz4, loss_dev);
  k_fc2_grad<<<1, F4, 0, s>>>(m->dz5, m->z4, n, G + OW5, G + OB5);
  // fc1: dW4[k][co] = sum_i a3[i][k] dz4[i][co], db4 = colsum(dz4), da3 = dz4 W4^T
  if ((e = igemm_wgrad(s, F4, K4, n, Dense{m->dz4, n, F4, F4}, Dense{m->a3, n, K4, K4}, G + OW4, m->part))) return e;
  if ((e = colsum(s, m->dz4, n, F4, m->part, G + OB4))) return e;
  if ((e = igemm<Dense, Dense, true>(s, n, K4, F4, Dense{m->dz4, n, F4, F4}, Dense{W + OW4, K4, F4, F4}, m->da, K4,
                                     nullptr)))
    return e;
  // conv3
  k_pool_relu_back<<<grid1((int64_t)n * PIX3 * C3), 256, 0, s>>>(m->da, m->i3, m->z3, n, 7, 7, C3, m->dzb);
  if ((e = igemm_wgrad(s, C3, K3, n * PIX3, Dense{m->dzb, n * PIX3, C3, C3}, ConvRows{m->a2, n, 7, 7, C2, 1},
                       G + OW3, m->part)))
    return e;
  if ((e = colsum(s, m->dzb, (int64_t)n * PIX3, C3, m->part, G + OB3))) return e;
  if ((e = igemm<ConvRows, ConvW, true>(s, n * PIX3, C2, 9 * C3, ConvRows{m->dzb, n, 7, 7, C3, -1},
                                        ConvW{W + OW3, C2, C3}, m->da, C2, nullptr)))
    return e;
  // conv2
  k_pool_relu_back<<<grid1((int64_t)n * PIX2 * C2), 256, 0, s>>>(m->da, m->i2, m->z2, n, 15, 15, C2, m->dzb);
  if ((e = igemm_wgrad(s, C2, K2, n * PIX2, Dense{m->dzb, n * PIX2, C2, C2}, ConvRows{m->a1, n, 15, 15, C1, 1},
                       G + OW2, m->part)))
    return e;
  if ((e = colsum(s, m->dzb, (int64_t)n * PIX2, C2, m->part, G + OB2))) return e;
  if ((e = igemm<ConvRows, ConvW, true>(s, n * PIX2, C1, 9 * C2, ConvRows{m->dzb, n, 15, 15, C2, -1},
                                        ConvW{W + OW2, C1, C2}, m->da, C1, nullptr)))
    return e;
  // conv1 (no input gradient)
  k_pool_relu_back<<<grid1((int64_t)n * PIX1 * C1), 256, 0, s>>>(m->da, m->i1, m->z1, n, S31, S31, C1, m->dzb);
  if ((e = igemm_wgrad(s, C1, K1, n * PIX1, Dense{m->dzb, n * PIX1, C1, C1}, Conv1Rows{m->xn, n, S31, S31},
                       G + OW1, m->part)))
    return e;
  if ((e = colsum(s, m->dzb, (int64_t)n * PIX1, C1, m->part, G + OB1))) return e;
  return cudaGetLastError();
}

void refresh_bf16(rb_model_s* m, cudaStream_t s) { k_to_bf16<<<grid1(NMASTER), 256, 0, s>>>(m->params, NMASTER, m->wbf); }

sfft_status_t fail(cudaError_t e, const char* where) {
  sfft::set_last_error((std::string(where) + ": " + cudaGetErrorString(e)).c_str());
  return SFFT_ERR_CUDA;
}

}  // namespace

extern "C" sfft_status_t rb_create(const int32_t* desc, rb_model_t* out) {
  if (!desc || !out || desc[0] < 1) return SFFT_ERR_ARG;
  *out = nullptr;
  if (desc[0] > 4096) return SFFT_ERR_UNSUPPORTED;   // GEMM grid rows: 961 * batch / 64 <= 65535
  rb_model_s* m = new (std::nothrow) rb_model_s();
  if (!m) return SFFT_ERR_NOMEM;
  const int B = desc[0];
  m->max_batch = B;
  bool ok = alloc(&m->params, NMASTER) && alloc(&m->grads, NMASTER) && alloc(&m->adam_m, NMASTER) &&
            alloc(&m->adam_v, NMASTER) && alloc(&m->wbf, NMASTER) && alloc(&m->xn, (size_t)B * PIX1 * 3) &&
            alloc(&m->a1, (size_t)B * PIX2 * C1) && alloc(&m->a2, (size_t)B * PIX3 * C2) &&
            alloc(&m->a3, (size_t)B * PIX4 * C3) &&
            alloc(&m->dzb, (size_t)B * PIX1 * C1) && alloc(&m->dz4, (size_t)B * F4) &&
            alloc(&m->z1, (size_t)B * PIX1 * C1) && alloc(&m->z2, (size_t)B * PIX2 * C2) &&
            alloc(&m->z3, (size_t)B * PIX3 * C3) && alloc(&m->z4, (size_t)B * F4) && alloc(&m->logit, (size_t)B) &&
            alloc(&m->dz5, (size_t)B) && alloc(&m->da, (size_t)B * PIX2 * C1 + B * K4) &&
            alloc(&m->i1, (size_t)B * PIX2 * C1) && alloc(&m->i2, (size_t)B * PIX3 * C2) &&
            alloc(&m->i3, (size_t)B * PIX4 * C3) && alloc(&m->part, (size_t)kMaxSplits * K4 * F4);
  if (!ok) {
    free_model(m);
    delete m;
    return SFFT_ERR_NOMEM;
  }
  // uniform He-style initialisation in the C-ABI layout, zero biases
  std::vector<float> abi(RB_NPARAM, 0.f);
  const int wsz[5] = {32 * 27, 64 * 288, 64 * 576, 128 * 576, 128};
  const int bsz[5] = {32, 64, 64, 128, 1};
  const int fan[5] = {27, 288, 576, 576, 128};
  size_t o = 0;
  for (int l = 0; l < 5; ++l) {
    const double lim = sqrt(6.0 / fan[l]);
    for (int i = 0; i < wsz[l]; ++i) abi[o + i] = (float)((2.0 * hash_uniform((uint64_t)desc[1], o + i) - 1.0) * lim);
    o += wsz[l] + bsz[l];
  }
  std::vector<float> master;
  abi_to_master(abi.data(), master);
  cudaError_t e = cudaMemcpy(m->params, master.data(), sizeof(float) * NMASTER, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->adam_m, 0, sizeof(float) * NMASTER);
  if (e == cudaSuccess) e = cudaMemset(m->adam_v, 0, sizeof(float) * NMASTER);
  if (e == cudaSuccess) e = cudaMemset(m->grads, 0, sizeof(float) * NMASTER);
  if (e == cudaSuccess) {
    refresh_bf16(m, nullptr);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    free_model(m);
    delete m;
    return fail(e, "rb_create");
  }
  *out = m;
  return SFFT_OK;
}

extern "C" sfft_status_t rb_destroy(rb_model_t m) {
  if (!m) return SFFT_ERR_ARG;
  free_model(m);
  delete m;
  return SFFT_OK;
}

extern "C" sfft_status_t rb_set_weights(rb_model_t m, const void* host_buf, size_t bytes) {
  if (!m || !host_buf || bytes != sizeof(float) * RB_NPARAM) return SFFT_ERR_ARG;
  std::vector<float> master;
  abi_to_master(static_cast<const float*>(host_buf), master);
  cudaError_t e = cudaMemcpy(m->params, master.data(), sizeof(float) * NMASTER, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(e, "rb_set_weights");
  refresh_bf16(m, nullptr);
  e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rb_set_weights");
}

static sfft_status_t get_vec(const float* dev, void* host_buf, size_t bytes, const char* where) {
  if (!dev || !host_buf || bytes != sizeof(float) * RB_NPARAM) return SFFT_ERR_ARG;
  std::vector<float> master(NMASTER);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(master.data(), dev, sizeof(float) * NMASTER, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(e, where);
  master_to_abi(master.data(), static_cast<float*>(host_buf));
  return SFFT_OK;
}

extern "C" sfft_status_t rb_get_weights(rb_model_t m, void* host_buf, size_t bytes) {
  return m ? get_vec(m->params, host_buf, bytes, "rb_get_weights") : SFFT_ERR_ARG;
}
extern "C" sfft_status_t rb_get_grads(rb_model_t m, void* host_buf, size_t bytes) {
  return m ? get_vec(m->grads, host_buf, bytes, "rb_get_grads") : SFFT_ERR_ARG;
}

extern "C" sfft_status_t rb_get_state(rb_model_t m, void* host_buf, size_t bytes, int64_t* step) {
  if (!m || !host_buf || bytes != 3 * sizeof(float) * RB_NPARAM) return SFFT_ERR_ARG;
  float* h = static_cast<float*>(host_buf);
  sfft_status_t st = get_vec(m->params, h, sizeof(float) * RB_NPARAM, "rb_get_state");
  if (st == SFFT_OK) st = get_vec(m->adam_m, h + RB_NPARAM, sizeof(float) * RB_NPARAM, "rb_get_state");
  if (st == SFFT_OK) st = get_vec(m->adam_v, h + 2 * RB_NPARAM, sizeof(float) * RB_NPARAM, "rb_get_state");
  if (st == SFFT_OK && step) *step = m->step;
  return st;
}

extern "C" sfft_status_t rb_set_state(rb_model_t m, const void* host_buf, size_t bytes, int64_t step) {
  if (!m || !host_buf || bytes != 3 * sizeof(float) * RB_NPARAM || step < 0) return SFFT_ERR_ARG;
  const float* h = static_cast<const float*>(host_buf);
  float* dst[3] = {m->params, m->adam_m, m->adam_v};
  for (int i = 0; i < 3; ++i) {
    std::vector<float> master;
    abi_to_master(h + (size_t)i * RB_NPARAM, master);
    cudaError_t e = cudaMemcpy(dst[i], master.data(), sizeof(float) * NMASTER, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(e, "rb_set_state");
  }
  m->step = step;
  refresh_bf16(m, nullptr);
  cudaError_t e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rb_set_state");
}

extern "C" sfft_status_t rb_logits(rb_model_t m, const float* stamps, int64_t n, float* logit, void* stream) {
  if (!m || (n > 0 && (!stamps || !logit)) || n < 0) return SFFT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int64_t i0 = 0; i0 < n; i0 += m->max_batch) {
    const int nb = (int)std::min<int64_t>(m->max_batch, n - i0);
    k_normalise<<<(3 * nb + 7) / 8, 256, 0, s>>>(stamps + i0 * 3 * PIX1, nb, m->xn);
    cudaError_t e = forward(m, nb, s, false);
    if (e == cudaSuccess) e = cudaMemcpyAsync(logit + i0, m->logit, sizeof(float) * nb, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(e, "rb_logits");
  }
  return SFFT_OK;
}

extern "C" sfft_status_t rb_score(rb_model_t m, const float* stamps, int64_t n, float* score, void* stream) {
  sfft_status_t st = rb_logits(m, stamps, n, score, stream);
  if (st != SFFT_OK || n == 0) return st;
  k_sigmoid<<<grid1(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(score, n, score);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rb_score");
}

extern "C" sfft_status_t rb_backward(rb_model_t m, const float* stamps, const float* labels, int64_t n,
                                     float* loss_dev, void* stream) {
  if (!m || !stamps || !labels || n < 1 || n > m->max_batch) return SFFT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = (int)n;
  k_normalise<<<(3 * nb + 7) / 8, 256, 0, s>>>(stamps, nb, m->xn);
  cudaError_t e = forward(m, nb, s, true);
  if (e == cudaSuccess) e = backward(m, nb, labels, loss_dev, s);
  return e == cudaSuccess ? SFFT_OK : fail(e, "rb_backward");
}

extern "C" sfft_status_t rb_train_step(rb_model_t m, const float* stamps, const float* labels, int64_t n, float lr,
                                       float* loss_dev, void* stream) {
  sfft_status_t st = rb_backward(m, stamps, labels, n, loss_dev, stream);
  if (st != SFFT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  m->step += 1;
  const float c1 = (float)(1.0 - pow(0.9, (double)m->step)), c2 = (float)(1.0 - pow(0.999, (double)m->step));
  k_adam<<<grid1(NMASTER), 256, 0, s>>>(m->params, m->grads, m->adam_m, m->adam_v, NMASTER, lr, c1, c2);
  refresh_bf16(m, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rb_train_step");
}
