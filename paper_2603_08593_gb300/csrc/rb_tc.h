// The stamp classifier's tensor-core inference convolutions (rb_conv_tc.cu):
// plane geometry of each layer's input and the launchers rb_cnn.cu calls.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rbtc {

// Input planes of a layer: CB blocks of 8 channels, each a plane of HP rows x
// WO columns of 16-byte records holding pixel (row - 1, column - 1); border
// records are zero.  Global layout [cb][stamp][HP * WO][8] (BF16).
struct Planes {
  int CB, HP, WO;
  size_t per_stamp_elems() const { return (size_t)HP * WO * 8; }
};
// normalised stamps: NHWC 31 x 31 x 3 BF16, then 5 zero values, so that a
// stamp is 5776 bytes and starts on a 16-byte boundary
constexpr int kXnStride = 2888;
constexpr Planes kP2{4, 18, 16};   // conv2 input: 15 x 15 x 32
constexpr Planes kP3{8, 10, 8};    // conv3 input: 7 x 7 x 64

// BF16 weight images of the three convolutions, one K = 16 slice per tap and
// pair of channel blocks (C_out rows x 16, K-major core matrices), built from
// the FP32 master weights in GEMM layout.  conv1 packs the three horizontal
// taps of a kernel row and the three input channels into one slice (9 of its
// 16 K entries; three slices); conv2 has 9 taps x 2 slices, conv3 9 x 4.
constexpr int kWImg1 = 3 * 1 * 16 * 32, kWImg2 = 9 * 2 * 16 * 64, kWImg3 = 9 * 4 * 16 * 64;

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
