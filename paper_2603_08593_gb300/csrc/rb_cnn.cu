// Stamp real-bogus classifier: BF16 tensor-core training and inference.
//
// Inference (rb_logits / rb_score) runs the three convolutions on the tcgen05
// tensor cores, each fused with its bias, ReLU and max-pool (rb_conv_tc.cu:
// channel-block planes, no FP32 pre-activations in memory).  Training keeps
// the FP32 pre-activations and pool indices its backward pass needs and runs
// on the path below.  Activations are NHWC.  Every training convolution is an
// implicit GEMM (rb_gemm.cuh: no im2col matrix is written) on mma.sync
// m16n8k16 BF16 with FP32 accumulation: forward  Z[pixel][co] = sum_k x(pixel + tap)[ci] W[k][co];
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
#include "rb_layers.cuh"
#include "rb_tc.h"

namespace {

// master parameter offsets (GEMM layout, floats)
constexpr int OW1 = 0, OB1 = OW1 + K1 * C1, OW2 = OB1 + C1, OB2 = OW2 + K2 * C2, OW3 = OB2 + C2,
              OB3 = OW3 + K3 * C3, OW4 = OB3 + C3, OB4 = OW4 + K4 * F4, OW5 = OB4 + F4, OB5 = OW5 + F4,
              NMASTER = OB5 + 1;

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
  // inference: BF16 weight images of the convolutions and the zero-bordered
  // channel-block planes of the conv2 and conv3 inputs; error word of the
  // tensor-core kernels (sticky: logits are NaN once a wait gave up)
  bf16 *img1 = nullptr, *img2 = nullptr, *img3 = nullptr, *p2 = nullptr, *p3 = nullptr;
  int* err = nullptr;
};

namespace {

void free_model(rb_model_s* m) {
  void* ptrs[] = {m->params, m->grads, m->adam_m, m->adam_v, m->wbf, m->xn,  m->a1,   m->a2,   m->a3,
                  m->dzb,    m->dz4,   m->z1,     m->z2,     m->z3,  m->z4, m->logit, m->dz5,  m->da,
                  m->part,   m->i1,    m->i2,     m->i3,  m->img1, m->img2, m->img3, m->p2,   m->p3,
                  m->err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

template <typename T>
bool alloc(T** p, size_t n) {
  return cudaMalloc((void**)p, sizeof(T) * (n > 0 ? n : 1)) == cudaSuccess;
}

// inference forward for n <= max_batch normalised stamps in m->xn: fused
// tcgen05 convolutions, then the dense layers; logits to m->logit
cudaError_t forward_infer(rb_model_s* m, int n, cudaStream_t s) {
  using rbg::Dense;
  const float* P = m->params;
  cudaError_t e;
  if ((e = rbtc::conv1_tc(m->xn, n, m->img1, P + OB1, m->p2, m->max_batch, m->err, s))) return e;
  if ((e = rbtc::conv2_tc(m->p2, n, m->img2, P + OB2, m->p3, m->max_batch, m->err, s))) return e;
  if ((e = rbtc::conv3_tc(m->p3, n, m->img3, P + OB3, m->a3, m->max_batch, m->err, s))) return e;
  if ((e = igemm<Dense, Dense, false>(s, n, F4, K4, Dense{m->a3, n, K4, K4}, Dense{m->wbf + OW4, K4, F4, F4}, m->z4,
                                      F4, P + OB4)))
    return e;
  k_fc2<<<(n * 32 + 255) / 256, 256, 0, s>>>(m->z4, P + OW5, P + OB5, n, m->logit, m->err);
  return cudaGetLastError();
}

// training forward for n <= max_batch normalised stamps in m->xn (FP32
// pre-activations and pool indices kept for the backward pass); logits to
// m->logit
cudaError_t forward(rb_model_s* m, int n, cudaStream_t s) {
  using rbg::ConvRows;
  using rbg::Conv1Rows;
  using rbg::Dense;
  const bf16* W = m->wbf;
  const float* P = m->params;
  cudaError_t e;
  // conv1 (3 -> 32): implicit GEMM over the 27 (padded 32) taps x channels
  if ((e = igemm<Conv1Rows, Dense, false>(s, n * PIX1, C1, K1, Conv1Rows{m->xn, n, S31, S31, rbtc::kXnStride},
                                          Dense{W + OW1, K1, C1, C1}, m->z1, C1, P + OB1)))
    return e;
  k_relu_pool<<<grid1((int64_t)n * PIX2 * C1), 256, 0, s>>>(m->z1, n, S31, S31, C1, m->a1, m->i1);
  // conv2 (32 -> 64)
  if ((e = igemm<ConvRows, Dense, false>(s, n * PIX2, C2, K2, ConvRows{m->a1, n, 15, 15, C1, 1},
                                         Dense{W + OW2, K2, C2, C2}, m->z2, C2, P + OB2)))
    return e;
  k_relu_pool<<<grid1((int64_t)n * PIX3 * C2), 256, 0, s>>>(m->z2, n, 15, 15, C2, m->a2, m->i2);
  // conv3 (64 -> 64)
  if ((e = igemm<ConvRows, Dense, false>(s, n * PIX3, C3, K3, ConvRows{m->a2, n, 7, 7, C2, 1},
                                         Dense{W + OW3, K3, C3, C3}, m->z3, C3, P + OB3)))
    return e;
  k_relu_pool<<<grid1((int64_t)n * PIX4 * C3), 256, 0, s>>>(m->z3, n, 7, 7, C3, m->a3, m->i3);
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
  k_fc2_grad<<<F4 / 8, 256, 0, s>>>(m->dz5, m->z4, n, G + OW5, G + OB5);
  // fc1: dW4[k][co] = sum_i a3[i][k] dz4[i][co], db4 = colsum(dz4), da3 = dz4 W4^T
  if ((e = igemm_wgrad(s, F4, K4, n, Dense{m->dz4, n, F4, F4}, Dense{m->a3, n, K4, K4}, G + OW4, m->part))) return e;
  if ((e = colsum(s, m->dz4, n, F4, m->part, G + OB4))) return e;
  if ((e = igemm<Dense, Dense, true>(s, n, K4, F4, Dense{m->dz4, n, F4, F4}, Dense{W + OW4, K4, F4, F4}, m->da, K4,
                                     nullptr)))
    return e;
  // conv3
  k_pool_relu_back<<<grid1((int64_t)n * PIX3 * C3 / 8), 256, 0, s>>>(m->da, m->i3, m->z3, n, 7, 7, C3, m->dzb);
  if ((e = igemm_wgrad(s, C3, K3, n * PIX3, Dense{m->dzb, n * PIX3, C3, C3}, ConvRows{m->a2, n, 7, 7, C2, 1},
                       G + OW3, m->part)))
    return e;
  if ((e = colsum(s, m->dzb, (int64_t)n * PIX3, C3, m->part, G + OB3))) return e;
  if ((e = igemm<ConvRows, ConvW, true>(s, n * PIX3, C2, 9 * C3, ConvRows{m->dzb, n, 7, 7, C3, -1},
                                        ConvW{W + OW3, C2, C3}, m->da, C2, nullptr)))
    return e;
  // conv2
  k_pool_relu_back<<<grid1((int64_t)n * PIX2 * C2 / 8), 256, 0, s>>>(m->da, m->i2, m->z2, n, 15, 15, C2, m->dzb);
  if ((e = igemm_wgrad(s, C2, K2, n * PIX2, Dense{m->dzb, n * PIX2, C2, C2}, ConvRows{m->a1, n, 15, 15, C1, 1},
                       G + OW2, m->part)))
    return e;
  if ((e = colsum(s, m->dzb, (int64_t)n * PIX2, C2, m->part, G + OB2))) return e;
  if ((e = igemm<ConvRows, ConvW, true>(s, n * PIX2, C1, 9 * C2, ConvRows{m->dzb, n, 15, 15, C2, -1},
                                        ConvW{W + OW2, C1, C2}, m->da, C1, nullptr)))
    return e;
  // conv1 (no input gradient)
  k_pool_relu_back<<<grid1((int64_t)n * PIX1 * C1 / 8), 256, 0, s>>>(m->da, m->i1, m->z1, n, S31, S31, C1, m->dzb);
  if ((e = igemm_wgrad(s, C1, K1, n * PIX1, Dense{m->dzb, n * PIX1, C1, C1},
                       Conv1Rows{m->xn, n, S31, S31, rbtc::kXnStride},
                       G + OW1, m->part)))
    return e;
  if ((e = colsum(s, m->dzb, (int64_t)n * PIX1, C1, m->part, G + OB1))) return e;
  return cudaGetLastError();
}

void refresh_bf16(rb_model_s* m, cudaStream_t s) {
  k_to_bf16<<<grid1(NMASTER), 256, 0, s>>>(m->params, NMASTER, m->wbf);
  rbtc::build_weight_images(m->params + OW1, m->params + OW2, m->params + OW3, m->img1, m->img2, m->img3, s);
}

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
            alloc(&m->adam_v, NMASTER) && alloc(&m->wbf, NMASTER) && alloc(&m->xn, (size_t)B * rbtc::kXnStride) &&
            alloc(&m->a1, (size_t)B * PIX2 * C1) && alloc(&m->a2, (size_t)B * PIX3 * C2) &&
            alloc(&m->a3, (size_t)B * PIX4 * C3) &&
            alloc(&m->dzb, (size_t)B * PIX1 * C1) && alloc(&m->dz4, (size_t)B * F4) &&
            alloc(&m->z1, (size_t)B * PIX1 * C1) && alloc(&m->z2, (size_t)B * PIX2 * C2) &&
            alloc(&m->z3, (size_t)B * PIX3 * C3) && alloc(&m->z4, (size_t)B * F4) && alloc(&m->logit, (size_t)B) &&
            alloc(&m->dz5, (size_t)B) && alloc(&m->da, (size_t)B * PIX2 * C1 + B * K4) &&
            alloc(&m->i1, (size_t)B * PIX2 * C1) && alloc(&m->i2, (size_t)B * PIX3 * C2) &&
            alloc(&m->i3, (size_t)B * PIX4 * C3) && alloc(&m->part, (size_t)kMaxSplits * K4 * F4) &&
            alloc(&m->img1, rbtc::kWImg1) && alloc(&m->img2, rbtc::kWImg2) && alloc(&m->img3, rbtc::kWImg3) &&
            alloc(&m->p2, (size_t)B * rbtc::kP2.per_stamp_elems()) &&
            alloc(&m->p3, (size_t)B * rbtc::kP3.per_stamp_elems()) && alloc(&m->err, 1);
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
  // the planes' borders stay zero: the convolutions write interiors only
  if (e == cudaSuccess) e = cudaMemset(m->p2, 0, sizeof(bf16) * (size_t)B * rbtc::kP2.per_stamp_elems());
  if (e == cudaSuccess) e = cudaMemset(m->p3, 0, sizeof(bf16) * (size_t)B * rbtc::kP3.per_stamp_elems());
  if (e == cudaSuccess) e = cudaMemset(m->err, 0, sizeof(int));
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
    k_normalise<<<nb, 96, 0, s>>>(stamps + i0 * 3 * PIX1, nb, m->xn, rbtc::kXnStride);
    cudaError_t e = forward_infer(m, nb, s);
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

extern "C" sfft_status_t rb_conv_layer(rb_model_t m, int32_t layer, const void* in, int64_t n, int64_t n_alloc,
                                       void* out, void* stream) {
  if (!m || layer < 1 || layer > 3 || n < 0 || n > n_alloc || n_alloc < 1 || n_alloc > (1 << 24))
    return SFFT_ERR_ARG;
  if (n == 0) return SFFT_OK;
  if (!in || !out || ((uintptr_t)in & 15) || ((uintptr_t)out & 15)) return SFFT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bf16* x = static_cast<const bf16*>(in);
  bf16* y = static_cast<bf16*>(out);
  const float* P = m->params;
  const int nn = (int)n, na = (int)n_alloc;
  cudaError_t e = layer == 1   ? rbtc::conv1_tc(x, nn, m->img1, P + OB1, y, na, m->err, s)
                  : layer == 2 ? rbtc::conv2_tc(x, nn, m->img2, P + OB2, y, na, m->err, s)
                               : rbtc::conv3_tc(x, nn, m->img3, P + OB3, y, na, m->err, s);
  return e == cudaSuccess ? SFFT_OK : fail(e, "rb_conv_layer");
}

extern "C" sfft_status_t rb_get_error(rb_model_t m, int32_t* flags) {
  if (!m || !flags) return SFFT_ERR_ARG;
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, m->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(e, "rb_get_error");
  *flags = v;
  return SFFT_OK;
}

extern "C" sfft_status_t rb_backward(rb_model_t m, const float* stamps, const float* labels, int64_t n,
                                     float* loss_dev, void* stream) {
  if (!m || !stamps || !labels || n < 1 || n > m->max_batch) return SFFT_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = (int)n;
  k_normalise<<<nb, 96, 0, s>>>(stamps, nb, m->xn, rbtc::kXnStride);
  cudaError_t e = forward(m, nb, s);
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
