// The paper's real-bogus classifier: a rotation-invariant network with
// residual blocks (Sec. 2.3.4 cites the DeepHiTS rotation-invariant framework
// and ResNet-18 residual connections; layer sizes are this library's reading).
//
// The normalised stamp (NHWC BF16) is presented in its four rotations by
// multiples of 90 degrees (rotation-major batch of 4 n) to one shared stack:
//   conv1  3 -> 32 + ReLU + 2 x 2 max-pool                 31 -> 15
//   res1   relu(p1 + conv_b(relu(conv_a(p1))))             32 channels, 15 x 15
//   conv2  32 -> 64 + ReLU + pool                          15 -> 7
//   res2   relu(p2 + conv_d(relu(conv_c(p2)))) + pool      64 channels, 7 -> 3
// and the four 576-feature vectors of a stamp are averaged (exact invariance
// under the rotations) before fc1 576 -> 128 + ReLU and fc2 128 -> 1.  Every
// convolution is an implicit GEMM on BF16 tensor-core MMA with FP32
// accumulation (rb_gemm.cuh); pre-activations are kept in FP32, activations
// fed to the next product in BF16, and the skip connections add the BF16
// activation that the branch itself consumed.  Training: BCE, backward through
// both paths of each block, Adam on FP32 master weights in GEMM layout.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "plan.h"
#include "rb.h"
#include "rb_layers.cuh"

namespace {

constexpr int NROT = 4;
constexpr int KA = 9 * C1, KC = 9 * C2;   // GEMM K of the residual convolutions (32 -> 32, 64 -> 64)

// master parameter offsets (GEMM layout, floats)
constexpr int QW1 = 0, QB1 = QW1 + K1 * C1, QWA = QB1 + C1, QBA = QWA + KA * C1, QWB = QBA + C1,
              QBB = QWB + KA * C1, QW2 = QBB + C1, QB2 = QW2 + K2 * C2, QWC = QB2 + C2, QBC = QWC + KC * C2,
              QWD = QBC + C2, QBD = QWD + KC * C2, QW4 = QBD + C2, QB4 = QW4 + K4 * F4, QW5 = QB4 + F4,
              QB5 = QW5 + F4, QMASTER = QB5 + 1;

// convolution layers in C-ABI order: (cin, cout, master weight offset, master bias offset)
struct ConvSpec { int cin, cout, ow, ob; };
constexpr ConvSpec kConv[6] = {{3, C1, QW1, QB1},  {C1, C1, QWA, QBA}, {C1, C1, QWB, QBB},
                               {C1, C2, QW2, QB2}, {C2, C2, QWC, QBC}, {C2, C2, QWD, QBD}};

// xr[r n + i] = the r-th counterclockwise quarter turn of xn[i]:
// r = 1: out(y, x) = in(x, 30 - y); r = 2: in(30 - y, 30 - x); r = 3: in(30 - x, y)
__global__ void k_rotate(const bf16* __restrict__ xn, int n, bf16* __restrict__ xr) {
  const int64_t total = (int64_t)NROT * n * PIX1 * 3;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % 3);
    const int64_t p = e / 3;
    const int pix = (int)(p % PIX1);
    const int64_t ri = p / PIX1;
    const int r = (int)(ri / n), i = (int)(ri % n);
    const int y = pix / S31, x = pix % S31;
    int sy = y, sx = x;
    if (r == 1) { sy = x; sx = S31 - 1 - y; }
    else if (r == 2) { sy = S31 - 1 - y; sx = S31 - 1 - x; }
    else if (r == 3) { sy = S31 - 1 - x; sx = y; }
    xr[e] = xn[((int64_t)i * PIX1 + sy * S31 + sx) * 3 + c];
  }
}

// a = bf16(relu(z))
__global__ void k_relu_bf16(const float* __restrict__ z, int64_t m, bf16* __restrict__ a) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    a[e] = __float2bfloat16(fmaxf(z[e], 0.f));
}

// z += skip (the BF16 activation the block's branch consumed)
__global__ void k_add_skip(float* __restrict__ z, const bf16* __restrict__ skip, int64_t m) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    z[e] += __bfloat162float(skip[e]);
}

// dz = (z > 0) ? d : 0, BF16
__global__ void k_relu_back(const float* __restrict__ d, const float* __restrict__ z, int64_t m,
                            bf16* __restrict__ dz) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    dz[e] = __float2bfloat16(z[e] > 0.f ? d[e] : 0.f);
}

// f[i][k] = mean over the four rotations of a3[r n + i][k] (rotations added in order 0..3)
__global__ void k_rot_mean(const bf16* __restrict__ a3, int n, float* __restrict__ f, bf16* __restrict__ fb) {
  const int64_t total = (int64_t)n * K4;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < NROT; ++r) s += __bfloat162float(a3[(int64_t)r * total + e]);
    s *= 0.25f;
    f[e] = s;
    fb[e] = __float2bfloat16(s);
  }
}

// da3[r n + i][k] = df[i][k] / 4
__global__ void k_rot_mean_back(const float* __restrict__ df, int n, float* __restrict__ da3) {
  const int64_t total = (int64_t)n * K4;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < NROT * total;
       e += (int64_t)gridDim.x * blockDim.x)
    da3[e] = 0.25f * df[e % total];
}

// d += g (BF16 gradient of the skip path)
__global__ void k_add_grad(float* __restrict__ d, const bf16* __restrict__ g, int64_t m) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    d[e] += __bfloat162float(g[e]);
}

// ---------------------------------------------------------------- layout conversion (host)
// C-ABI order: w1 b1 wa ba wb bb w2 b2 wc bc wd bd ([cout][cin][3][3] and [cout]),
// w4 [128][576] (input index channel * 9 + row * 3 + column), b4, w5 [1][128], b5
void abi_to_master(const float* a, std::vector<float>& m) {
  m.assign(QMASTER, 0.f);
  size_t o = 0;
  for (const ConvSpec& L : kConv) {
    const float* w = a + o;
    for (int co = 0; co < L.cout; ++co)
      for (int ci = 0; ci < L.cin; ++ci)
        for (int t = 0; t < 9; ++t) m[L.ow + (t * L.cin + ci) * L.cout + co] = w[(co * L.cin + ci) * 9 + t];
    o += (size_t)L.cout * L.cin * 9;
    for (int co = 0; co < L.cout; ++co) m[L.ob + co] = a[o + co];
    o += L.cout;
  }
  for (int f = 0; f < F4; ++f)
    for (int c = 0; c < C3; ++c)
      for (int p = 0; p < PIX4; ++p) m[QW4 + (p * C3 + c) * F4 + f] = a[o + (size_t)f * K4 + c * PIX4 + p];
  o += (size_t)F4 * K4;
  for (int f = 0; f < F4; ++f) m[QB4 + f] = a[o + f];
  o += F4;
  for (int f = 0; f < F4; ++f) m[QW5 + f] = a[o + f];
  m[QB5] = a[o + F4];
}

void master_to_abi(const float* m, float* a) {
  size_t o = 0;
  for (const ConvSpec& L : kConv) {
    float* w = a + o;
    for (int co = 0; co < L.cout; ++co)
      for (int ci = 0; ci < L.cin; ++ci)
        for (int t = 0; t < 9; ++t) w[(co * L.cin + ci) * 9 + t] = m[L.ow + (t * L.cin + ci) * L.cout + co];
    o += (size_t)L.cout * L.cin * 9;
    for (int co = 0; co < L.cout; ++co) a[o + co] = m[L.ob + co];
    o += L.cout;
  }
  for (int f = 0; f < F4; ++f)
    for (int c = 0; c < C3; ++c)
      for (int p = 0; p < PIX4; ++p) a[o + (size_t)f * K4 + c * PIX4 + p] = m[QW4 + (p * C3 + c) * F4 + f];
  o += (size_t)F4 * K4;
  for (int f = 0; f < F4; ++f) a[o + f] = m[QB4 + f];
  o += F4;
  for (int f = 0; f < F4; ++f) a[o + f] = m[QW5 + f];
  a[o + F4] = m[QB5];
}

}  // namespace

struct rbri_model_s {
  int max_batch = 0;
  int64_t step = 0;
  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  bf16* wbf = nullptr;
  // activations for 4 max_batch rotated stamps (FP32 pre-activations, BF16 activations)
  bf16 *xn = nullptr, *xr = nullptr, *a1 = nullptr, *ra = nullptr, *r1 = nullptr, *a2 = nullptr, *rc = nullptr,
       *a3 = nullptr, *fb = nullptr, *dz4 = nullptr, *dzA = nullptr, *dzB = nullptr;
  float *z1 = nullptr, *za = nullptr, *zb = nullptr, *z2 = nullptr, *zc = nullptr, *zd = nullptr, *f = nullptr,
        *z4 = nullptr, *logit = nullptr, *dz5 = nullptr, *da = nullptr, *part = nullptr;
  uint8_t *i1 = nullptr, *i2 = nullptr, *i3 = nullptr;
};

namespace {

void free_model(rbri_model_s* m) {
  void* ptrs[] = {m->params, m->grads, m->adam_m, m->adam_v, m->wbf, m->xn, m->xr, m->a1, m->ra, m->r1, m->a2,
                  m->rc, m->a3, m->fb, m->dz4, m->dzA, m->dzB, m->z1, m->za, m->zb, m->z2, m->zc, m->zd, m->f,
                  m->z4, m->logit, m->dz5, m->da, m->part, m->i1, m->i2, m->i3};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

template <typename T>
bool alloc(T** p, size_t n) {
  return cudaMalloc((void**)p, sizeof(T) * (n > 0 ? n : 1)) == cudaSuccess;
}

// forward for n normalised stamps in m->xn; logits to m->logit
cudaError_t forward(rbri_model_s* m, int n, cudaStream_t s, bool keep_idx) {
  using rbg::ConvRows;
  using rbg::Conv1Rows;
  using rbg::Dense;
  const bf16* W = m->wbf;
  const float* P = m->params;
  const int n4 = NROT * n;
  cudaError_t e;
  k_rotate<<<grid1((int64_t)n4 * PIX1 * 3), 256, 0, s>>>(m->xn, n, m->xr);
  // conv1 + ReLU + pool
  if ((e = igemm<Conv1Rows, Dense, false>(s, n4 * PIX1, C1, K1, Conv1Rows{m->xr, n4, S31, S31, 3 * PIX1},
                                          Dense{W + QW1, K1, C1, C1}, m->z1, C1, P + QB1)))
    return e;
  k_relu_pool<<<grid1((int64_t)n4 * PIX2 * C1), 256, 0, s>>>(m->z1, n4, S31, S31, C1, m->a1, keep_idx ? m->i1 : nullptr);
  // res1
  const int64_t m1 = (int64_t)n4 * PIX2 * C1;
  if ((e = igemm<ConvRows, Dense, false>(s, n4 * PIX2, C1, KA, ConvRows{m->a1, n4, 15, 15, C1, 1},
                                         Dense{W + QWA, KA, C1, C1}, m->za, C1, P + QBA)))
    return e;
  k_relu_bf16<<<grid1(m1), 256, 0, s>>>(m->za, m1, m->ra);
  if ((e = igemm<ConvRows, Dense, false>(s, n4 * PIX2, C1, KA, ConvRows{m->ra, n4, 15, 15, C1, 1},
                                         Dense{W + QWB, KA, C1, C1}, m->zb, C1, P + QBB)))
    return e;
  k_add_skip<<<grid1(m1), 256, 0, s>>>(m->zb, m->a1, m1);
  k_relu_bf16<<<grid1(m1), 256, 0, s>>>(m->zb, m1, m->r1);
  // conv2 + ReLU + pool
  if ((e = igemm<ConvRows, Dense, false>(s, n4 * PIX2, C2, K2, ConvRows{m->r1, n4, 15, 15, C1, 1},
                                         Dense{W + QW2, K2, C2, C2}, m->z2, C2, P + QB2)))
    return e;
  k_relu_pool<<<grid1((int64_t)n4 * PIX3 * C2), 256, 0, s>>>(m->z2, n4, 15, 15, C2, m->a2, keep_idx ? m->i2 : nullptr);
  // res2 + pool
  const int64_t m2 = (int64_t)n4 * PIX3 * C2;
  if ((e = igemm<ConvRows, Dense, false>(s, n4 * PIX3, C2, KC, ConvRows{m->a2, n4, 7, 7, C2, 1},
                                         Dense{W + QWC, KC, C2, C2}, m->zc, C2, P + QBC)))
    return e;
  k_relu_bf16<<<grid1(m2), 256, 0, s>>>(m->zc, m2, m->rc);
  if ((e = igemm<ConvRows, Dense, false>(s, n4 * PIX3, C2, KC, ConvRows{m->rc, n4, 7, 7, C2, 1},
                                         Dense{W + QWD, KC, C2, C2}, m->zd, C2, P + QBD)))
    return e;
  k_add_skip<<<grid1(m2), 256, 0, s>>>(m->zd, m->a2, m2);
  k_relu_pool<<<grid1((int64_t)n4 * PIX4 * C2), 256, 0, s>>>(m->zd, n4, 7, 7, C2, m->a3, keep_idx ? m->i3 : nullptr);
  // rotation average, dense head
  k_rot_mean<<<grid1((int64_t)n * K4), 256, 0, s>>>(m->a3, n, m->f, m->fb);
  if ((e = igemm<Dense, Dense, false>(s, n, F4, K4, Dense{m->fb, n, K4, K4}, Dense{W + QW4, K4, F4, F4}, m->z4, F4,
                                      P + QB4)))
    return e;
  k_fc2<<<(n * 32 + 255) / 256, 256, 0, s>>>(m->z4, P + QW5, P + QB5, n, m->logit);
  return cudaGetLastError();
}

// weight gradient, bias gradient and (optionally) input gradient of one 3 x 3 convolution
cudaError_t conv_back(rbri_model_s* m, cudaStream_t s, int n4, int hw, int cin, int cout, const bf16* dz,
                      const bf16* x, int ow, int ob, float* dx) {
  using rbg::ConvRows;
  using rbg::Dense;
  float* G = m->grads;
  const int pix = hw * hw;
  cudaError_t e;
  if ((e = igemm_wgrad(s, cout, 9 * cin, n4 * pix, Dense{dz, n4 * pix, cout, cout},
                       ConvRows{x, n4, hw, hw, cin, 1}, G + ow, m->part)))
    return e;
  if ((e = colsum(s, dz, (int64_t)n4 * pix, cout, m->part, G + ob))) return e;
  if (dx)
    return igemm<ConvRows, ConvW, true>(s, n4 * pix, cin, 9 * cout, ConvRows{dz, n4, hw, hw, cout, -1},
                                        ConvW{m->wbf + ow, cin, cout}, dx, cin, nullptr);
  return cudaSuccess;
}

cudaError_t backward(rbri_model_s* m, int n, const float* labels, float* loss_dev, cudaStream_t s) {
  using rbg::Conv1Rows;
  using rbg::Dense;
  const bf16* W = m->wbf;
  float* G = m->grads;
  const int n4 = NROT * n;
  cudaError_t e;
  cudaMemsetAsync(G, 0, sizeof(float) * QMASTER, s);
  k_bce_head<<<1, 1024, 0, s>>>(m->logit, labels, n, m->z4, m->params + QW5, m->dz5, m->dz4, loss_dev);
  k_fc2_grad<<<F4 / 8, 256, 0, s>>>(m->dz5, m->z4, n, G + QW5, G + QB5);
  // fc1: dW4 = sum_i dz4[i] f[i], db4, df = dz4 W4^T
  if ((e = igemm_wgrad(s, F4, K4, n, Dense{m->dz4, n, F4, F4}, Dense{m->fb, n, K4, K4}, G + QW4, m->part))) return e;
  if ((e = colsum(s, m->dz4, n, F4, m->part, G + QB4))) return e;
  float* df = m->f;   // the FP32 features are not needed any more
  if ((e = igemm<Dense, Dense, true>(s, n, K4, F4, Dense{m->dz4, n, F4, F4}, Dense{W + QW4, K4, F4, F4}, df, K4,
                                     nullptr)))
    return e;
  // rotation average and the last pool
  k_rot_mean_back<<<grid1((int64_t)n4 * K4), 256, 0, s>>>(df, n, m->da);
  k_pool_relu_back<<<grid1((int64_t)n4 * PIX3 * C2 / 8), 256, 0, s>>>(m->da, m->i3, m->zd, n4, 7, 7, C2, m->dzA);
  // res2: zd = conv_d(rc) + a2
  const int64_t m2 = (int64_t)n4 * PIX3 * C2;
  if ((e = conv_back(m, s, n4, 7, C2, C2, m->dzA, m->rc, QWD, QBD, m->da))) return e;
  k_relu_back<<<grid1(m2), 256, 0, s>>>(m->da, m->zc, m2, m->dzB);
  if ((e = conv_back(m, s, n4, 7, C2, C2, m->dzB, m->a2, QWC, QBC, m->da))) return e;
  k_add_grad<<<grid1(m2), 256, 0, s>>>(m->da, m->dzA, m2);   // the skip path
  // conv2
  k_pool_relu_back<<<grid1((int64_t)n4 * PIX2 * C2 / 8), 256, 0, s>>>(m->da, m->i2, m->z2, n4, 15, 15, C2, m->dzA);
  if ((e = conv_back(m, s, n4, 15, C1, C2, m->dzA, m->r1, QW2, QB2, m->da))) return e;
  // res1: r1 = relu(zb), zb = conv_b(ra) + a1
  const int64_t m1 = (int64_t)n4 * PIX2 * C1;
  k_relu_back<<<grid1(m1), 256, 0, s>>>(m->da, m->zb, m1, m->dzA);
  if ((e = conv_back(m, s, n4, 15, C1, C1, m->dzA, m->ra, QWB, QBB, m->da))) return e;
  k_relu_back<<<grid1(m1), 256, 0, s>>>(m->da, m->za, m1, m->dzB);
  if ((e = conv_back(m, s, n4, 15, C1, C1, m->dzB, m->a1, QWA, QBA, m->da))) return e;
  k_add_grad<<<grid1(m1), 256, 0, s>>>(m->da, m->dzA, m1);   // the skip path
  // conv1 (no input gradient)
  k_pool_relu_back<<<grid1((int64_t)n4 * PIX1 * C1 / 8), 256, 0, s>>>(m->da, m->i1, m->z1, n4, S31, S31, C1, m->dzA);
  if ((e = igemm_wgrad(s, C1, K1, n4 * PIX1, Dense{m->dzA, n4 * PIX1, C1, C1},
                       Conv1Rows{m->xr, n4, S31, S31, 3 * PIX1},
                       G + QW1, m->part)))
    return e;
  if ((e = colsum(s, m->dzA, (int64_t)n4 * PIX1, C1, m->part, G + QB1))) return e;
  return cudaGetLastError();
}

void refresh_bf16(rbri_model_s* m, cudaStream_t s) {
  k_to_bf16<<<grid1(QMASTER), 256, 0, s>>>(m->params, QMASTER, m->wbf);
}

sfft_status_t fail(cudaError_t e, const char* where) {
  sfft::set_last_error((std::string(where) + ": " + cudaGetErrorString(e)).c_str());
  return SFFT_ERR_CUDA;
}

}  // namespace

extern "C" sfft_status_t rbri_create(const int32_t* desc, rbri_model_t* out) {
  if (!desc || !out || desc[0] < 1) return SFFT_ERR_ARG;
  *out = nullptr;
  if (desc[0] > 2048) return SFFT_ERR_UNSUPPORTED;   // GEMM grid rows: 4 * 961 * batch / 128 <= 65535
  rbri_model_s* m = new (std::nothrow) rbri_model_s();
  if (!m) return SFFT_ERR_NOMEM;
  const int B = desc[0];
  const size_t B4 = (size_t)NROT * B;
  m->max_batch = B;
  bool ok = alloc(&m->params, QMASTER) && alloc(&m->grads, QMASTER) && alloc(&m->adam_m, QMASTER) &&
            alloc(&m->adam_v, QMASTER) && alloc(&m->wbf, QMASTER) && alloc(&m->xn, (size_t)B * PIX1 * 3) &&
            alloc(&m->xr, B4 * PIX1 * 3) && alloc(&m->a1, B4 * PIX2 * C1) && alloc(&m->ra, B4 * PIX2 * C1) &&
            alloc(&m->r1, B4 * PIX2 * C1) && alloc(&m->a2, B4 * PIX3 * C2) && alloc(&m->rc, B4 * PIX3 * C2) &&
            alloc(&m->a3, B4 * K4) && alloc(&m->fb, (size_t)B * K4) && alloc(&m->dz4, (size_t)B * F4) &&
            alloc(&m->dzA, B4 * PIX1 * C1) && alloc(&m->dzB, B4 * PIX2 * C1) && alloc(&m->z1, B4 * PIX1 * C1) &&
            alloc(&m->za, B4 * PIX2 * C1) && alloc(&m->zb, B4 * PIX2 * C1) && alloc(&m->z2, B4 * PIX2 * C2) &&
            alloc(&m->zc, B4 * PIX3 * C2) && alloc(&m->zd, B4 * PIX3 * C2) && alloc(&m->f, (size_t)B * K4) &&
            alloc(&m->z4, (size_t)B * F4) && alloc(&m->logit, (size_t)B) && alloc(&m->dz5, (size_t)B) &&
            alloc(&m->da, B4 * PIX2 * C1) && alloc(&m->i1, B4 * PIX2 * C1) && alloc(&m->i2, B4 * PIX3 * C2) &&
            alloc(&m->i3, B4 * PIX4 * C2) && alloc(&m->part, (size_t)kMaxSplits * K4 * F4);
  if (!ok) {
    free_model(m);
    delete m;
    return SFFT_ERR_NOMEM;
  }
  // uniform He-style initialisation in the C-ABI layout, zero biases
  std::vector<float> abi(RBRI_NPARAM, 0.f);
  size_t o = 0;
  auto fill = [&](size_t nw, int fan, size_t nb) {
    const double lim = sqrt(6.0 / fan);
    for (size_t i = 0; i < nw; ++i) abi[o + i] = (float)((2.0 * hash_uniform((uint64_t)desc[1], o + i) - 1.0) * lim);
    o += nw + nb;
  };
  for (const ConvSpec& L : kConv) fill((size_t)L.cout * L.cin * 9, 9 * L.cin, L.cout);
  fill((size_t)F4 * K4, K4, F4);
  fill(F4, F4, 1);
  std::vector<float> master;
  abi_to_master(abi.data(), master);
  cudaError_t e = cudaMemcpy(m->params, master.data(), sizeof(float) * QMASTER, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->adam_m, 0, sizeof(float) * QMASTER);
  if (e == cudaSuccess) e = cudaMemset(m->adam_v, 0, sizeof(float) * QMASTER);
  if (e == cudaSuccess) e = cudaMemset(m->grads, 0, sizeof(float) * QMASTER);
  if (e == cudaSuccess) {
    refresh_bf16(m, nullptr);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    free_model(m);
    delete m;
    return fail(e, "rbri_create");
  }
  *out = m;
  return SFFT_OK;
}

extern "C" sfft_status_t rbri_destroy(rbri_model_t m) {
  if (!m) return SFFT_ERR_ARG;
  free_model(m);
  delete m;
  return SFFT_OK;
}

extern "C" sfft_status_t rbri_set_weights(rbri_model_t m, const void* host_buf, size_t bytes) {
  if (!m || !host_buf || bytes != sizeof(float) * RBRI_NPARAM) return SFFT_ERR_ARG;
  std::vector<float> master;
  abi_to_master(static_cast<const float*>(host_buf), master);
  cudaError_t e = cudaMemcpy(m->params, master.data(), sizeof(float) * QMASTER, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(e, "rbri_set_weights");
  refresh_bf16(m, nullptr);
  e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rbri_set_weights");
}

static sfft_status_t get_vec(const float* dev, void* host_buf, size_t bytes, const char* where) {
  if (!host_buf || bytes != sizeof(float) * RBRI_NPARAM) return SFFT_ERR_ARG;
  std::vector<float> master(QMASTER);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(master.data(), dev, sizeof(float) * QMASTER, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(e, where);
  master_to_abi(master.data(), static_cast<float*>(host_buf));
  return SFFT_OK;
}

extern "C" sfft_status_t rbri_get_weights(rbri_model_t m, void* host_buf, size_t bytes) {
  return m ? get_vec(m->params, host_buf, bytes, "rbri_get_weights") : SFFT_ERR_ARG;
}
extern "C" sfft_status_t rbri_get_grads(rbri_model_t m, void* host_buf, size_t bytes) {
  return m ? get_vec(m->grads, host_buf, bytes, "rbri_get_grads") : SFFT_ERR_ARG;
}

extern "C" sfft_status_t rbri_get_state(rbri_model_t m, void* host_buf, size_t bytes, int64_t* step) {
  if (!m || !host_buf || !step || bytes != 3 * sizeof(float) * RBRI_NPARAM) return SFFT_ERR_ARG;
  float* h = static_cast<float*>(host_buf);
  const float* src[3] = {m->params, m->adam_m, m->adam_v};
  for (int i = 0; i < 3; ++i) {
    const sfft_status_t st = get_vec(src[i], h + (size_t)i * RBRI_NPARAM, sizeof(float) * RBRI_NPARAM, "rbri_get_state");
    if (st != SFFT_OK) return st;
  }
  *step = m->step;
  return SFFT_OK;
}

extern "C" sfft_status_t rbri_set_state(rbri_model_t m, const void* host_buf, size_t bytes, int64_t step) {
  if (!m || !host_buf || bytes != 3 * sizeof(float) * RBRI_NPARAM || step < 0) return SFFT_ERR_ARG;
  const float* h = static_cast<const float*>(host_buf);
  float* dst[3] = {m->params, m->adam_m, m->adam_v};
  for (int i = 0; i < 3; ++i) {
    std::vector<float> master;
    abi_to_master(h + (size_t)i * RBRI_NPARAM, master);
    cudaError_t e = cudaMemcpy(dst[i], master.data(), sizeof(float) * QMASTER, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(e, "rbri_set_state");
  }
  m->step = step;
  refresh_bf16(m, nullptr);
  cudaError_t e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rbri_set_state");
}

extern "C" sfft_status_t rbri_logits(rbri_model_t m, const float* stamps, int64_t n, float* logit, void* stream) {
  if (!m || (n > 0 && (!stamps || !logit)) || n < 0) return SFFT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int64_t i0 = 0; i0 < n; i0 += m->max_batch) {
    const int nb = (int)std::min<int64_t>(m->max_batch, n - i0);
    k_normalise<<<nb, 96, 0, s>>>(stamps + i0 * 3 * PIX1, nb, m->xn, 3 * PIX1);
    cudaError_t e = forward(m, nb, s, false);
    if (e == cudaSuccess) e = cudaMemcpyAsync(logit + i0, m->logit, sizeof(float) * nb, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail(e, "rbri_logits");
  }
  return SFFT_OK;
}

extern "C" sfft_status_t rbri_score(rbri_model_t m, const float* stamps, int64_t n, float* score, void* stream) {
  sfft_status_t st = rbri_logits(m, stamps, n, score, stream);
  if (st != SFFT_OK || n == 0) return st;
  k_sigmoid<<<grid1(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(score, n, score);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rbri_score");
}

extern "C" sfft_status_t rbri_backward(rbri_model_t m, const float* stamps, const float* labels, int64_t n,
                                       float* loss_dev, void* stream) {
  if (!m || !stamps || !labels || n < 1 || n > m->max_batch) return SFFT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = (int)n;
  k_normalise<<<nb, 96, 0, s>>>(stamps, nb, m->xn, 3 * PIX1);
  cudaError_t e = forward(m, nb, s, true);
  if (e == cudaSuccess) e = backward(m, nb, labels, loss_dev, s);
  return e == cudaSuccess ? SFFT_OK : fail(e, "rbri_backward");
}

extern "C" sfft_status_t rbri_train_step(rbri_model_t m, const float* stamps, const float* labels, int64_t n, float lr,
                                         float* loss_dev, void* stream) {
  sfft_status_t st = rbri_backward(m, stamps, labels, n, loss_dev, stream);
  if (st != SFFT_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  m->step += 1;
  const float c1 = (float)(1.0 - pow(0.9, (double)m->step)), c2 = (float)(1.0 - pow(0.999, (double)m->step));
  k_adam<<<grid1(QMASTER), 256, 0, s>>>(m->params, m->grads, m->adam_m, m->adam_v, QMASTER, lr, c1, c2);
  refresh_bf16(m, s);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : fail(e, "rbri_train_step");
}
