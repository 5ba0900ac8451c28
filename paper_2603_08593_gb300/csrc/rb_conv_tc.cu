// Inference convolutions of the stamp classifier on the tcgen05 tensor cores:
// each of the three 3 x 3 'same' convolutions, with its bias, ReLU and 2 x 2
// max-pool, in one kernel that reads BF16 activations and writes the next
// layer's BF16 activations (no FP32 pre-activation image reaches memory).
//
// Layout.  A layer's input is held, per stamp, as channel-block planes: for
// each block of 8 channels a plane of HP rows x WO columns of 16-byte records
// (8 BF16 channels), where plane row r and column c hold the input pixel
// (r - 1, c - 1) and every other record (the border) is zero.  WO is a power
// of two at least W + 1, and HP = H + 2 rounded up to an even number.  The
// convolution's output slots are the same HP x WO grid: slot m = y WO + x is
// output pixel (y, x), and for the tap (dy, dx) it reads the record at slot
// m + (dy + 1) WO + dx + 1 of the plane, i.e. the input pixel (y + dy, x + dx)
// or the zero border; slots with y >= H or x >= W compute values nobody reads.
// So the A operand of one MMA (M = 128 consecutive slots x K = 16 channels of
// one tap) is a plain strided view of the planes: core matrices of 8 slots x
// 8 channels are 128 contiguous bytes (stride byte offset 128) and the second
// 8 channels are the next channel block's plane (leading byte offset = the
// distance between planes).  No im2col matrix is built anywhere.  The B
// operand (the tap's weights, N = C_out rows x K = 16) is a K-major image in
// shared memory, copied once per launch from an image built when the
// weights change.  conv1 has 3 input channels only: its records hold, for the
// input pixel row of the plane row, the 3 channels of three horizontally
// adjacent pixels (9 of 16 K entries, the rest zero), so one MMA covers a
// whole kernel row and a tile takes 3 MMAs instead of 9.
//
// A CTA takes S stamps at a time (S HP WO is a multiple of 128): it copies
// their planes to shared memory (conv1 builds them from the normalised NHWC
// stamp), issues per 128-slot tile 9 taps x (channel blocks / 2) MMAs into
// tensor memory, TACC tiles per round, and its four warps read the
// accumulators back (tcgen05.ld, one slot per thread), take the 2 x 2 maximum
// with the neighbouring slots (lane shuffles, or through shared memory when a
// warp holds one image row), add the bias, apply the ReLU and store the
// pooled BF16 values: into the next layer's planes, or (after the last
// convolution) into the NHWC [n][3][3][64] activations of the dense layers.
// Pool windows never straddle a tile: a tile is 128 / WO whole image rows and
// HP is even.  Every wait is bounded; a wait that gives up sets the model's
// error word and the CTA leaves after draining its MMAs.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "bulk.cuh"
#include "common.cuh"
#include "rb_tc.h"
#include "umma_common.cuh"

namespace rbtc {

using bf16 = __nv_bfloat16;
using sfft::elect_one;
using sfft::instr_desc;
using sfft::kMaxSpin;
using sfft::mbar_arrive_expect_tx;
using sfft::mbar_init;
using sfft::mbar_try_wait;
using sfft::smem_desc_kn;
using sfft::smem_u32;

constexpr int kThreads = 128;

__device__ __forceinline__ bool wait_bounded(uint64_t* bar, unsigned parity) {
  for (int it = 0; it < kMaxSpin; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// 32 consecutive FP32 accumulator columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
               "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
               "[%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                 "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                 "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                 "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}


// Per-layer geometry.  Input planes: CB channel blocks, HP x WO records per
// stamp, an H x H image; S stamps per group (S HP WO a multiple of 128);
// N output channels; NTAP MMA taps per tile of K = 16 per channel-block pair;
// TACC tiles accumulated per round in TCOLS tensor-memory columns.  Output:
// the next layer's planes (CBO x HPO x WOO) or, after conv3, NHWC rows.
template <int LAYER>
struct Cfg;
template <>
struct Cfg<1> {
  static constexpr int CB = 2, HP = 34, WO = 32, H = 31, S = 2, N = 32, NTAP = 3, TACC = 8, TCOLS = 256;
  static constexpr int HPO = 18, WOO = 16;
  static constexpr bool NHWC = false;
};
template <>
struct Cfg<2> {
  static constexpr int CB = 4, HP = 18, WO = 16, H = 15, S = 4, N = 64, NTAP = 9, TACC = 4, TCOLS = 256;
  static constexpr int HPO = 10, WOO = 8;
  static constexpr bool NHWC = false;
};
template <>
struct Cfg<3> {
  static constexpr int CB = 8, HP = 10, WO = 8, H = 7, S = 8, N = 64, NTAP = 9, TACC = 5, TCOLS = 512;
  static constexpr int HPO = 0, WOO = 0;
  static constexpr bool NHWC = true;
};

template <int LAYER>
struct Geo {
  using C = Cfg<LAYER>;
  static constexpr int HPWO = C::HP * C::WO;
  static constexpr int T = C::S * HPWO / 128;              // tiles per group
  static constexpr int KS = C::CB / 2;                     // K = 16 slices per tap
  static constexpr int PAD = 2 * C::WO + 8;                // records past the last slot a tap may read
  static constexpr int STK = C::S * HPWO + PAD;            // records per channel-block stack
  static constexpr int IMG = C::NTAP * KS * 32 * C::N;     // weight-image bytes
  static constexpr int STAGE = LAYER == 1 ? C::S * kXnStride * 2 : 0;   // conv1: normalised stamps (bytes)
  static constexpr int XCH = C::WO == 32 ? 16 * 128 * 4 : 0;        // cross-warp pool exchange (bytes)
  static constexpr size_t SMEM = (size_t)C::CB * STK * 16 + IMG + XCH + STAGE;
  static_assert((C::S * HPWO) % 128 == 0, "whole tiles per group");
  static_assert(C::HP % 2 == 0 && 128 % C::WO == 0 && (128 / C::WO) % 2 == 0, "pool windows inside a tile");
  static_assert(C::TACC * C::N <= C::TCOLS && STK < 16384, "tensor memory and descriptor ranges");
  static_assert((C::CB * STK * 16) % 128 == 0 && IMG % 128 == 0, "shared-memory alignment");
};

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ uint32_t bf_bits(bf16 v) { return (uint32_t)__bfloat16_as_ushort(v); }

// conv1 planes of the group's stamps s0 .. s0 + ns - 1 from the normalised
// stamps staged in shared memory (kXnStride values each); record (r, c) of
// block 0 holds channels 0-2 of input pixels (r - 1, c - 2), (r - 1, c - 1)
// and channels 0-1 of (r - 1, c); block 1 holds channel 2 of (r - 1, c);
// zero outside the image and for stamps past ns.
__device__ __forceinline__ void build_conv1_planes(int ns, uint4* planes, const bf16* sb) {
  using G = Geo<1>;
  for (int idx = threadIdx.x; idx < Cfg<1>::S * G::HPWO; idx += kThreads) {
    const int s = idx / G::HPWO, rem = idx - s * G::HPWO, r = rem >> 5, c = rem & 31;
    uint32_t k[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) k[i] = 0;
    const int row = r - 1;
    if (s < ns && row >= 0 && row < 31) {
#pragma unroll
      for (int dxi = 0; dxi < 3; ++dxi) {
        const int col = c - 2 + dxi;
        if (col >= 0 && col < 31) {
          const bf16* p = sb + s * kXnStride + (row * 31 + col) * 3;
#pragma unroll
          for (int ci = 0; ci < 3; ++ci) k[dxi * 3 + ci] = bf_bits(p[ci]);
        }
      }
    }
    planes[idx] = make_uint4(k[0] | (k[1] << 16), k[2] | (k[3] << 16), k[4] | (k[5] << 16), k[6] | (k[7] << 16));
    planes[G::STK + idx] = make_uint4(k[8], 0u, 0u, 0u);
  }
}

// 2 x 2 max of one 32-column chunk over the four slots of a pool window as a
// reduce-scatter: the horizontal partner (lane ^ 1) and the vertical partner
// (lane ^ 16 for WO = 16, lane ^ 8 for WO = 8, the same lane of warp ^ 1 for
// WO = 32, through `xs`) each keep half of what they hold, so every thread
// ends with the maximum of 8 channels: 32 ch + 16 h + 8 v + i, i = 0 .. 7.
template <int WO>
__device__ __forceinline__ void pool_chunk(const float (&v)[32], float (&q)[8], float* xs, int& h, int& vb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  h = lane & 1;
  float r[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const float send = h ? v[i] : v[16 + i], keep = h ? v[16 + i] : v[i];
    r[i] = fmaxf(keep, __shfl_xor_sync(0xffffffffu, send, 1));
  }
  if constexpr (WO == 32) {
    vb = warp & 1;
#pragma unroll
    for (int i = 0; i < 16; ++i) xs[i * 128 + threadIdx.x] = r[i];
    __syncthreads();
    const int partner = threadIdx.x ^ 32;
#pragma unroll
    for (int i = 0; i < 8; ++i) q[i] = fmaxf(vb ? r[8 + i] : r[i], xs[(8 * vb + i) * 128 + partner]);
    __syncthreads();
  } else {
    constexpr int X = WO == 16 ? 16 : 8;
    vb = (lane / X) & 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float send = vb ? r[i] : r[8 + i], keep = vb ? r[8 + i] : r[i];
      q[i] = fmaxf(keep, __shfl_xor_sync(0xffffffffu, send, X));
    }
  }
}

// Copies of group g's input into shared memory, counted on `bar` (thread 0):
// conv1 the normalised stamps, the other layers their channel-block planes.
template <int LAYER>
__device__ __forceinline__ void issue_group_copy(const bf16* in, int g, int n, int n_alloc, uint4* planes,
                                                 uint8_t* stage, uint64_t* bar) {
  using C = Cfg<LAYER>;
  using G = Geo<LAYER>;
  const int s0 = g * C::S, ns = min(C::S, n - s0);
  if constexpr (LAYER == 1) {
    const unsigned bytes = (unsigned)(ns * kXnStride * 2);
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(stage, in + (size_t)s0 * kXnStride, bytes, bar);
  } else {
    const unsigned bytes = (unsigned)(ns * G::HPWO * 16);
    mbar_arrive_expect_tx(bar, (unsigned)C::CB * bytes);
    for (int cb = 0; cb < C::CB; ++cb)
      bulk_g2s(planes + cb * G::STK, in + ((size_t)cb * n_alloc + s0) * G::HPWO * 8, bytes, bar);
  }
}

// One convolution layer (see the file comment).  in: conv1 the normalised
// stamps ([n][kXnStride]), else the layer's input planes ([cb][n_alloc][HP WO]
// records); out: the next layer's planes (same n_alloc) or NHWC [n][3][3][64].
// The next group's copy is issued as soon as its buffer is free: for conv1
// right after the planes are built from the staged stamps (it overlaps the
// MMAs and the epilogue), for the other layers after the last round's MMAs
// (it overlaps that round's epilogue; the remainder round goes first so that
// the last round is a full one).
template <int LAYER>
__global__ void __launch_bounds__(kThreads, 1)
k_conv_tc(const bf16* __restrict__ in, int n, int n_alloc, const bf16* __restrict__ img,
          const float* __restrict__ bias, bf16* __restrict__ out, int* __restrict__ err) {
  using C = Cfg<LAYER>;
  using G = Geo<LAYER>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint4* planes = reinterpret_cast<uint4*>(smem);
  uint8_t* bimg = smem + (size_t)C::CB * G::STK * 16;
  float* xs = reinterpret_cast<float*>(bimg + G::IMG);
  uint8_t* stage = bimg + G::IMG + G::XCH;
  __shared__ uint64_t load_bar, mma_bar, w_bar;
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ngroups = (n + C::S - 1) / C::S;
  if (tid == 0) {
    mbar_init(&load_bar, 1);
    mbar_init(&mma_bar, 1);
    mbar_init(&w_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the stacks' pads are read only for output slots nobody keeps; zero them
  for (int i = tid; i < C::CB * G::PAD; i += kThreads)
    planes[(i / G::PAD) * G::STK + C::S * G::HPWO + i % G::PAD] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "n"(C::TCOLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;
  const uint32_t lane_off = (uint32_t)(32 * warp) << 16;

  // this thread's epilogue channels (pool_chunk's reduce-scatter): 32 ch +
  // 16 h + 8 v + i; their biases stay in registers
  const int h_me = lane & 1;
  const int v_me = C::WO == 32 ? (warp & 1) : ((lane / (C::WO == 16 ? 16 : 8)) & 1);
  float breg[C::N / 32][8];
#pragma unroll
  for (int ch = 0; ch < C::N / 32; ++ch)
#pragma unroll
    for (int i = 0; i < 8; ++i) breg[ch][i] = __ldg(bias + 32 * ch + 16 * h_me + 8 * v_me + i);

  if (tid == 0) {
    mbar_arrive_expect_tx(&w_bar, (unsigned)G::IMG);
    bulk_g2s(bimg, img, (unsigned)G::IMG, &w_bar);
    if (blockIdx.x < ngroups) issue_group_copy<LAYER>(in, blockIdx.x, n, n_alloc, planes, stage, &load_bar);
  }
  bool load_pending = (int)blockIdx.x < ngroups, mma_pending = false;
  bool ok = __syncthreads_and(wait_bounded(&w_bar, 0));
  const bool w_pending = !ok;
  unsigned lphase = 0, mphase = 0;
  constexpr uint32_t idesc = instr_desc(1, C::N);
  const uint64_t bdesc0 = smem_desc_kn(smem_u32(bimg), 16 * C::N, 128);
  const uint64_t adesc0 = smem_desc_kn(smem_u32(planes), G::STK * 16, 128);

  for (int g = blockIdx.x; ok && g < ngroups; g += gridDim.x) {
    const int s0 = g * C::S, ns = min(C::S, n - s0), gn = g + (int)gridDim.x;
    // ---- the group's input
    ok = __syncthreads_and(wait_bounded(&load_bar, lphase));
    if (!ok) break;
    load_pending = false;
    lphase ^= 1u;
    if constexpr (LAYER == 1) {
      build_conv1_planes(ns, planes, reinterpret_cast<const bf16*>(stage));
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (gn < ngroups) {   // the stage is free: fetch the next group's stamps
        if (tid == 0) issue_group_copy<LAYER>(in, gn, n, n_alloc, planes, stage, &load_bar);
        load_pending = true;
      }
    }
    // ---- rounds of up to TACC tiles (the remainder first): MMAs into tensor
    // memory, then the epilogue
    for (int t0 = 0; t0 < G::T;) {
      const int nt = (t0 == 0 && G::T % C::TACC) ? G::T % C::TACC : C::TACC;
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int tt = 0; tt < nt; ++tt) {
          const uint32_t dcol = tbase + (uint32_t)(tt * C::N);
#pragma unroll
          for (int j = 0; j < C::NTAP; ++j) {
            const int off = C::NTAP == 9 ? (j / 3) * C::WO + j % 3 : j * C::WO + 1;   // record of the tap
#pragma unroll
            for (int ks = 0; ks < G::KS; ++ks) {
              const uint64_t a = adesc0 + (uint64_t)(2 * ks * G::STK + (t0 + tt) * 128 + off);
              const uint64_t b = bdesc0 + (uint64_t)((j * G::KS + ks) * 2 * C::N);
              mma_bf16(dcol, a, b, idesc, (j | ks) ? 1u : 0u);
            }
          }
        }
        mma_commit(&mma_bar);
      }
      mma_pending = true;
      ok = __syncthreads_and(wait_bounded(&mma_bar, mphase));
      if (!ok) break;
      mma_pending = false;
      mphase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (LAYER != 1 && t0 + nt == G::T && gn < ngroups) {   // planes no longer read: fetch the next group's
        if (tid == 0) issue_group_copy<LAYER>(in, gn, n, n_alloc, planes, stage, &load_bar);
        load_pending = true;
      }
      for (int tt = 0; tt < nt; ++tt) {
        const int m = (t0 + tt) * 128 + 32 * warp + lane;   // this thread's slot (tensor-memory lane)
        const int R = m / C::WO, s = R / C::HP, yo = (R % C::HP) >> 1, xo = (m % C::WO) >> 1;
        const bool keep = s < ns && yo < C::H / 2 && xo < C::H / 2;
#pragma unroll
        for (int ch = 0; ch < C::N / 32; ++ch) {
          float v[32], q[8];
          int h, vb;
          tmem_ld32(tbase + lane_off + (uint32_t)(tt * C::N + 32 * ch), v);
          pool_chunk<C::WO>(v, q, xs, h, vb);
          const int c0 = 32 * ch + 16 * h + 8 * vb;
          float o[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) o[i] = fmaxf(q[i] + breg[ch][i], 0.f);
          const uint4 rec = make_uint4(pack2(o[0], o[1]), pack2(o[2], o[3]), pack2(o[4], o[5]), pack2(o[6], o[7]));
          if (keep) {
            size_t at;   // record index of the output
            if constexpr (C::NHWC)
              at = (((size_t)(s0 + s) * 9 + yo * 3 + xo) * 64 + c0) / 8;
            else
              at = ((size_t)(c0 / 8) * n_alloc + (s0 + s)) * (C::HPO * C::WOO) + (yo + 1) * C::WOO + xo + 1;
            reinterpret_cast<uint4*>(out)[at] = rec;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      t0 += nt;
    }
  }

  // ---- teardown: a wait that gave up flags the error; copies or MMAs still
  // in flight are waited for (bounded) before the shared and tensor memory go
  if (tid == 0) {
    if (!ok) atomicOr(err, 1);
    if (w_pending) wait_bounded(&w_bar, 0);
    if (load_pending) wait_bounded(&load_bar, lphase);
    if (mma_pending) wait_bounded(&mma_bar, mphase);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(C::TCOLS) : "memory");
}

// Weight images: element (j, ks, kc, co, e) of a layer with N output channels
// sits at (((j KS + ks) 2 + kc) N + co) 8 + e and holds the weight of input
// channel (2 ks + kc) 8 + e of tap j (conv1: K entry k = 8 kc + e, k < 9, is
// tap (j, k / 3), channel k % 3; entries k >= 9 are zero).  Masters in GEMM
// layout [(tap cin + ci)][cout].
__global__ void k_weight_images(const float* __restrict__ w1, const float* __restrict__ w2,
                                const float* __restrict__ w3, bf16* __restrict__ img1, bf16* __restrict__ img2,
                                bf16* __restrict__ img3) {
  const int total = kWImg1 + kWImg2 + kWImg3;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int i = idx, N, KS, cin;
    const float* w;
    bf16* img;
    if (i < kWImg1) {
      N = 32, KS = 1, cin = 3, w = w1, img = img1;
    } else if ((i -= kWImg1) < kWImg2) {
      N = 64, KS = 2, cin = 32, w = w2, img = img2;
    } else {
      i -= kWImg2;
      N = 64, KS = 4, cin = 64, w = w3, img = img3;
    }
    const int e = i & 7, co = (i >> 3) % N, kc = (i / (8 * N)) & 1, jks = i / (16 * N);
    const int ks = jks % KS, j = jks / KS;
    float v;
    if (cin == 3) {
      const int k = 8 * kc + e;   // kernel row j, column k / 3, channel k % 3: GEMM row 9 j + k
      v = k < 9 ? w[(j * 9 + k) * 32 + co] : 0.f;
    } else {
      v = w[(j * cin + (2 * ks + kc) * 8 + e) * N + co];
    }
    img[i] = __float2bfloat16(v);
  }
}

template <int LAYER>
cudaError_t launch(const bf16* in, int n, int n_alloc, const bf16* img, const float* bias, bf16* out, int* err,
                   cudaStream_t s) {
  using C = Cfg<LAYER>;
  using G = Geo<LAYER>;
  if (n <= 0) return cudaSuccess;
  static int grid_cap = 0;
  if (grid_cap == 0) {
    // CTAs per SM: as many as the SM's shared memory holds (the carveout set
    // to its maximum), at most as many as share its 512 tensor-memory columns
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<LAYER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_conv_tc<LAYER>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    int dev = 0, sms = 0, smem_sm = 0, reserved = 0;
    cudaFuncAttributes fa{};
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_conv_tc<LAYER>);
    if (e != cudaSuccess) return e;
    const int per_cta = (int)G::SMEM + (int)fa.sharedSizeBytes + reserved;
    const int occ = std::max(1, std::min(smem_sm / per_cta, 512 / C::TCOLS));
    grid_cap = occ * sms;
  }
  const int ngroups = (n + C::S - 1) / C::S;
  k_conv_tc<LAYER><<<std::min(ngroups, grid_cap), kThreads, G::SMEM, s>>>(in, n, n_alloc, img, bias, out, err);
  return cudaGetLastError();
}

cudaError_t build_weight_images(const float* w1, const float* w2, const float* w3, bf16* img1, bf16* img2,
                                bf16* img3, cudaStream_t s) {
  k_weight_images<<<(kWImg1 + kWImg2 + kWImg3 + 255) / 256, 256, 0, s>>>(w1, w2, w3, img1, img2, img3);
  return cudaGetLastError();
}

cudaError_t conv1_tc(const bf16* xn, int n, const bf16* img1, const float* b1, bf16* p2, int n_alloc, int* err,
                     cudaStream_t s) {
  return launch<1>(xn, n, n_alloc, img1, b1, p2, err, s);
}
cudaError_t conv2_tc(const bf16* p2, int n, const bf16* img2, const float* b2, bf16* p3, int n_alloc, int* err,
                     cudaStream_t s) {
  return launch<2>(p2, n, n_alloc, img2, b2, p3, err, s);
}
cudaError_t conv3_tc(const bf16* p3, int n, const bf16* img3, const float* b3, bf16* a3, int n_alloc, int* err,
                     cudaStream_t s) {
  return launch<3>(p3, n, n_alloc, img3, b3, a3, err, s);
}

}  // namespace rbtc
