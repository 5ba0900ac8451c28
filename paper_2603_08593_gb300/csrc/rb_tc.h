// The stamp classifier's tensor-core inference convolutions (rb_conv_tc.cu):
// plane geometry of each layer's input and the launchers rb_cnn.cu calls.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rbtc {

// Input planes of conv2 and conv3: CB blocks of 8 channels; the image padded
// with a zero border (padded pixel (r, c) = pixel (r - 1, c - 1)) and split by
// the parities of r and c into four WS x WS sub-planes of 16-byte records
// (record (r >> 1, c >> 1) of sub-plane 2 (r & 1) + (c & 1)); every record
// that holds no pixel is zero.  Memory layout [cb][parity][stamp][WS][WS][8]
// BF16, stamps 0 .. n_alloc - 1.
struct Planes {
  int CB, WS;
  size_t per_stamp_elems() const { return (size_t)CB * 4 * WS * WS * 8; }
};
// normalised stamps: NHWC 31 x 31 x 3 BF16, then 5 zero values, so that a
// stamp is 5776 bytes and starts on a 16-byte boundary
constexpr int kXnStride = 2888;
constexpr Planes kP2{4, 8};   // conv2 input: 15 x 15 x 32
constexpr Planes kP3{8, 4};   // conv3 input: 7 x 7 x 64

// BF16 weight images of the three convolutions (K-major core matrices, one
// K = 16 slice per MMA), built from the FP32 master weights in GEMM layout:
// conv1 4 row offsets x 128 (4 window positions x 32 channels) x 16, conv2
// 9 taps x 2 slices x 64 x 16, conv3 9 x 4 x 64 x 16 values.
constexpr int kWImg1 = 4 * 128 * 16, kWImg2 = 9 * 2 * 16 * 64, kWImg3 = 9 * 4 * 16 * 64;

// Build the three weight images (one launch).  w1, w2, w3: master weights in
// GEMM layout [(tap * cin + ci)][cout] (conv1 with its 32 padded rows).
cudaError_t build_weight_images(const float* w1, const float* w2, const float* w3, __nv_bfloat16* img1,
                                __nv_bfloat16* img2, __nv_bfloat16* img3, cudaStream_t s);

// conv1 + bias + ReLU + pool: xn [n][kXnStride] -> conv2 planes p2
// (n_alloc stamps per channel block); conv2 ... -> conv3 planes p3; conv3 ...
// -> a3 NHWC [n][3][3][64].  err: device word that a wait that gives up sets.
cudaError_t conv1_tc(const __nv_bfloat16* xn, int n, const __nv_bfloat16* img1, const float* b1, __nv_bfloat16* p2,
                     int n_alloc, int* err, cudaStream_t s);
cudaError_t conv2_tc(const __nv_bfloat16* p2, int n, const __nv_bfloat16* img2, const float* b2, __nv_bfloat16* p3,
                     int n_alloc, int* err, cudaStream_t s);
cudaError_t conv3_tc(const __nv_bfloat16* p3, int n, const __nv_bfloat16* img3, const float* b3, __nv_bfloat16* a3,
                     int n_alloc, int* err, cudaStream_t s);

}  // namespace rbtc
