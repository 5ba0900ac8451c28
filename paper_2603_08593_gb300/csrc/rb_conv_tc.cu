// Inference convolutions of the stamp classifier on the tcgen05 tensor cores:
// each of the three 3 x 3 'same' convolutions, with its bias, ReLU and 2 x 2
// max-pool, in one kernel that reads BF16 activations and writes the next
// layer's BF16 activations (no FP32 pre-activation image reaches memory).
//
// Layout.  A layer's input is held as parity-split channel-block planes.  Pad
// the H x H image with a zero border (padded pixel (r, c) = input pixel
// (r - 1, c - 1)) and split the padded pixels by the parities of r and c into
// four sub-planes of WS x WS records (16-byte records of 8 BF16 channels):
// record (r >> 1, c >> 1) of sub-plane 2 (r & 1) + (c & 1).  Every record
// that is no input pixel is zero.  The MMA rows are pool windows, not
// pixels: window (wy, wx) covers the outputs (2 wy + a, 2 wx + b), a, b in
// {0, 1}, and for window position (a, b) and tap (dy, dx) it reads padded
// pixel (2 wy + a + dy + 1, 2 wx + b + dx + 1), that is record
// (wy + i, wx + j) of sub-plane (p, q) with a + dy + 1 = 2 i + p and
// b + dx + 1 = 2 j + q.  For fixed (a, b, dy, dx) consecutive windows read
// consecutive records, so the A operand of one MMA (M = 128 windows x K = 16
// channels) is a plain strided view of shared memory: core matrices of 8
// windows x 8 channels are 128 contiguous bytes (stride byte offset 128),
// the other 8 channels sit in the next channel block (leading byte offset).
// Each window position accumulates into its own N columns of tensor memory,
// so one thread (tensor-memory lane = window) holds all four outputs of its
// window: the 2 x 2 max-pool, bias and ReLU are register arithmetic.  No
// im2col matrix is built anywhere.  The B operand (a tap's weights, N = C_out
// x K = 16) is a K-major image in shared memory, copied once per launch from
// an image built when the weights change.
//
// conv1 has 3 input channels.  Its record for padded row r and window column
// wx holds the 3 channels of the four input pixels (r - 1, 2 wx - 1 .. 2 wx + 2)
// that the window's two output columns and three kernel columns touch (12 of
// 16 K entries), so the records are split by row parity only, and the A
// operand for padded-row offset ro = a + dy + 1 (0 .. 3) is shared by every
// window position and kernel row that reads it: one MMA per offset with
// N = 4 positions x 32 channels, whose weight image holds, for position
// (a, b), the weights of kernel row ro - a and columns e - b for pixel e (zero
// where that tap does not exist).  4 MMAs of N = 128 per tile instead of 36
// of N = 32: the MMAs run at the tensor cores' arithmetic rate instead of the
// shared-memory operand rate.  conv1 expands these records in shared memory
// from the normalised NHWC stamps.
//
// Windows of stamp s occupy rows s WS^2 + wy WS + wx of a group of S stamps
// (the sub-planes of the group's stamps are contiguous); windows with wy or
// wx beyond the pooled size compute values nobody reads.  The kernel is
// persistent and warp-specialised: warps 0-3 read the accumulators back
// (tcgen05.ld) and write the pooled outputs, warp 4 issues the MMAs (one
// elected lane), warp 5 copies the inputs (bulk copies), and for conv1 warps
// 6-9 expand the staged stamps into planes.  Input buffers and accumulator
// slots are double-buffered and handed over by mbarriers, so copies, plane
// expansion, MMAs and epilogues of consecutive groups overlap.  Every wait is
// bounded; a wait that gives up raises the CTA's abort flag and the model's
// error word, and every role leaves after draining what it issued.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "bulk.cuh"
#include "common.cuh"
#include "rb.h"
#include "rb_tc.h"
#include "umma_common.cuh"

namespace rbtc {

using bf16 = __nv_bfloat16;
using sfft::instr_desc;
using sfft::kMaxSpin;
using sfft::mbar_arrive;
using sfft::mbar_arrive_expect_tx;
using sfft::mbar_init;
using sfft::mbar_try_wait;
using sfft::smem_desc_kn;
using sfft::smem_u32;
using sfft::wait_phase;

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

// Four groups of 32 FP32 accumulator columns of this thread's tensor-memory
// lane, starting at taddr + q * stride (q = 0 .. 3), with one wait for all
__device__ __forceinline__ void tmem_ld4x32(uint32_t taddr, uint32_t stride, float (&v)[128]) {
  uint32_t r[128];
  asm volatile(
      "{\n"
      ".reg .b32 a1, a2, a3;\n"
      "add.u32 a1, %128, %129;\n"
      "add.u32 a2, a1, %129;\n"
      "add.u32 a3, a2, %129;\n"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%128];\n"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, "
      "%46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [a1];\n"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%64, %65, %66, %67, %68, %69, %70, %71, %72, %73, %74, %75, %76, %77, "
      "%78, %79, %80, %81, %82, %83, %84, %85, %86, %87, %88, %89, %90, %91, %92, %93, %94, %95}, [a2];\n"
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%96, %97, %98, %99, %100, %101, %102, %103, %104, %105, %106, %107, "
      "%108, %109, %110, %111, %112, %113, %114, %115, %116, %117, %118, %119, %120, %121, %122, %123, %124, %125, "
      "%126, %127}, [a3];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      "}\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
        "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
        "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
        "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63]), "=r"(r[64]),
        "=r"(r[65]), "=r"(r[66]), "=r"(r[67]), "=r"(r[68]), "=r"(r[69]), "=r"(r[70]), "=r"(r[71]), "=r"(r[72]),
        "=r"(r[73]), "=r"(r[74]), "=r"(r[75]), "=r"(r[76]), "=r"(r[77]), "=r"(r[78]), "=r"(r[79]), "=r"(r[80]),
        "=r"(r[81]), "=r"(r[82]), "=r"(r[83]), "=r"(r[84]), "=r"(r[85]), "=r"(r[86]), "=r"(r[87]), "=r"(r[88]),
        "=r"(r[89]), "=r"(r[90]), "=r"(r[91]), "=r"(r[92]), "=r"(r[93]), "=r"(r[94]), "=r"(r[95]), "=r"(r[96]),
        "=r"(r[97]), "=r"(r[98]), "=r"(r[99]), "=r"(r[100]), "=r"(r[101]), "=r"(r[102]), "=r"(r[103]),
        "=r"(r[104]), "=r"(r[105]), "=r"(r[106]), "=r"(r[107]), "=r"(r[108]), "=r"(r[109]), "=r"(r[110]),
        "=r"(r[111]), "=r"(r[112]), "=r"(r[113]), "=r"(r[114]), "=r"(r[115]), "=r"(r[116]), "=r"(r[117]),
        "=r"(r[118]), "=r"(r[119]), "=r"(r[120]), "=r"(r[121]), "=r"(r[122]), "=r"(r[123]), "=r"(r[124]),
        "=r"(r[125]), "=r"(r[126]), "=r"(r[127])
      : "r"(taddr), "r"(stride));
#pragma unroll
  for (int i = 0; i < 128; ++i) v[i] = __uint_as_float(r[i]);
}

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

// Per-layer geometry.  CB input channel blocks, NPAR parity sub-planes (conv1:
// row parity only) of WS x WS records (= window grid), PH pooled outputs per
// side (valid windows), S stamps per group, N output channels, NTAP taps per
// window position (conv1: the 4 row offsets, each one MMA over all positions);
// WSO the sub-plane width of the output planes.
template <int LAYER>
struct Cfg;
template <>
struct Cfg<1> {
  static constexpr int CB = 2, NPAR = 2, WS = 16, PH = 15, S = 2, N = 32, NTAP = 4, WSO = 8;
  static constexpr bool NHWC = false;
};
template <>
struct Cfg<2> {
  static constexpr int CB = 4, NPAR = 4, WS = 8, PH = 7, S = 4, N = 64, NTAP = 9, WSO = 4;
  static constexpr bool NHWC = false;
};
template <>
struct Cfg<3> {
  static constexpr int CB = 8, NPAR = 4, WS = 4, PH = 3, S = 8, N = 64, NTAP = 9, WSO = 0;
  static constexpr bool NHWC = true;
};

template <int LAYER>
struct Geo {
  using C = Cfg<LAYER>;
  static constexpr int SP = C::WS * C::WS;                  // records per sub-plane and stamp
  static constexpr int GW = C::S * SP;                      // windows (MMA rows) per group
  static constexpr int T = GW / 128;                        // tiles per group
  static constexpr int KS = C::CB / 2;                      // K = 16 slices per tap
  static constexpr int CBS = C::NPAR * GW;                  // records per channel block
  static constexpr int PAD = (C::WS + 8) & ~7;              // >= WS + 1 records a tap may read past the end
  static constexpr int BUF = C::CB * CBS + PAD;             // records per input buffer
  static constexpr int ACC = 4 * C::N;                      // accumulator columns per tile
  static constexpr int NSLOT = 512 / ACC;                   // accumulator slots
  static constexpr int NMMA = LAYER == 1 ? 4 * C::N : C::N;   // N of one MMA
  static constexpr int IMG = C::NTAP * KS * 32 * NMMA;      // weight-image bytes
  static constexpr int STAGE = LAYER == 1 ? C::S * kXnStride * 2 : 0;   // conv1: normalised stamps (bytes)
  static constexpr int NWARP = LAYER == 1 ? 10 : 6;
  static constexpr size_t SMEM_USED = 2 * (size_t)BUF * 16 + IMG + 2 * (size_t)STAGE;
  // requested shared memory: at least enough that no two CTAs share an SM
  // (each allocates all 512 tensor-memory columns)
  static constexpr size_t SMEM = SMEM_USED > 120 * 1024 ? SMEM_USED : 120 * 1024;
  static_assert(GW % 128 == 0 && CBS < 16384, "whole tiles per group, descriptor range");
  static_assert(NSLOT >= 2 && SMEM <= 227 * 1024, "double buffering");
  static_assert((BUF * 16) % 128 == 0 && IMG % 128 == 0 && STAGE % 16 == 0, "shared-memory alignment");
};

constexpr int WARP_MMA = 4, WARP_COPY = 5, WARP_BUILD = 6;

// Time attribution (compile with -DRBTC_WAIT_PROFILE): lane 0 of every warp
// adds the cycles its role spends in each wait and work phase to a per-layer
// device array that rb_debug_conv_waits reads.  The default build compiles
// none of it.
enum ConvTime {
  CT_CTA = 0,         // warp 0: the CTA's whole run
  CT_COPY_EMPTY,      // copy warp: an input buffer (or stamp stage) to be released
  CT_BUILD_STAGE,     // conv1 builders: staged stamps to land
  CT_BUILD_EMPTY,     // conv1 builders: an input buffer to be released by the MMAs
  CT_BUILD_WORK,      // conv1 builders: expanding records
  CT_MMA_FULL,        // MMA warp: an input buffer to be filled
  CT_MMA_ACC_EMPTY,   // MMA warp: an accumulator slot to be released
  CT_MMA_ISSUE,       // MMA warp: issuing a tile's MMAs
  CT_EPI_FULL,        // epilogue warps: a tile's accumulators
  CT_EPI_WORK,        // epilogue warps: reading, pooling and storing a tile
  CT_NKIND
};
#ifdef RBTC_WAIT_PROFILE
__device__ unsigned long long g_conv_time[3][CT_NKIND];
#define CT_T0() long long ct_t0_ = clock64()
#define CT_ACC(kind) ct_acc_[kind] += clock64() - ct_t0_
#else
#define CT_T0() \
  do {          \
  } while (0)
#define CT_ACC(kind) \
  do {               \
  } while (0)
#endif

// conv1 records of the group's stamps (ns of S) in input buffer `dst` from
// the staged normalised stamps: for padded row r < 32 and window column wx,
// K entry 3 e + c (e = 0 .. 3, c = 0 .. 2) is channel c of input pixel
// (r - 1, 2 wx - 1 + e), entries 12 .. 15 zero; block 0 holds entries 0-7,
// block 1 entries 8-15.  Zero outside the image and for stamps past ns.  `t`
// counts the 128 building threads.
__device__ __forceinline__ void build_conv1(int ns, uint4* dst, const bf16* sb, int t) {
  using G = Geo<1>;
  for (int idx = t; idx < Cfg<1>::S * 512; idx += 128) {
    const int s = idx >> 9, r = (idx >> 4) & 31, wx = idx & 15;
    uint32_t k[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) k[i] = 0;
    const int row = r - 1;
    if (s < ns && row >= 0 && row < 31) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = 2 * wx - 1 + e;
        if (col >= 0 && col < 31) {
          const bf16* p = sb + s * kXnStride + (row * 31 + col) * 3;
#pragma unroll
          for (int c = 0; c < 3; ++c) k[3 * e + c] = bf_bits(p[c]);
        }
      }
    }
    const int at = (r & 1) * G::GW + s * G::SP + (r >> 1) * Cfg<1>::WS + wx;
    dst[at] = make_uint4(k[0] | (k[1] << 16), k[2] | (k[3] << 16), k[4] | (k[5] << 16), k[6] | (k[7] << 16));
    dst[G::CBS + at] = make_uint4(k[8] | (k[9] << 16), k[10] | (k[11] << 16), 0u, 0u);
  }
}

// Bulk copies of group g's input (thread 0 of the copy warp): conv1 the
// normalised stamps into `stage`, the other layers their planes ([cb][parity]
// [n_alloc][SP] records in memory, [cb][parity][S][SP] in `buf`).
template <int LAYER>
__device__ __forceinline__ void issue_group_copy(const bf16* in, int g, int n, int n_alloc, uint4* buf,
                                                 uint8_t* stage, uint64_t* bar) {
  using C = Cfg<LAYER>;
  using G = Geo<LAYER>;
  const int s0 = g * C::S, ns = min(C::S, n - s0);
  if constexpr (LAYER == 1) {
    const unsigned bytes = (unsigned)(ns * kXnStride * 2);
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(stage, in + (size_t)s0 * kXnStride, bytes, bar);
  } else {
    const unsigned bytes = (unsigned)(ns * G::SP * 16);
    mbar_arrive_expect_tx(bar, (unsigned)(C::NPAR * C::CB) * bytes);
    for (int cp = 0; cp < C::NPAR * C::CB; ++cp)   // (channel block, parity)
      bulk_g2s(buf + (cp / C::NPAR) * G::CBS + (cp % C::NPAR) * G::GW, in + ((size_t)cp * n_alloc + s0) * G::SP * 8,
               bytes, bar);
  }
}

// One convolution layer (see the file comment).  in: conv1 the normalised
// stamps ([n][kXnStride]), else the layer's input planes; out: the next
// layer's planes ([cb][parity][n_alloc][WSO^2] records) or, after conv3, NHWC
// [n][3][3][64].
template <int LAYER>
__global__ void __launch_bounds__(32 * Geo<LAYER>::NWARP, 1)
k_conv_tc(const bf16* __restrict__ in, int n, int n_alloc, const bf16* __restrict__ img,
          const float* __restrict__ bias, bf16* __restrict__ out, int* __restrict__ err) {
  using C = Cfg<LAYER>;
  using G = Geo<LAYER>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint4* buf0 = reinterpret_cast<uint4*>(smem);                 // input buffers 0 and 1
  uint8_t* bimg = smem + 2 * (size_t)G::BUF * 16;
  uint8_t* stage0 = bimg + G::IMG;                             // conv1: staged stamps 0 and 1
  __shared__ uint64_t in_full[2], in_empty[2], st_full[2], st_empty[2], acc_full[G::NSLOT], acc_empty[G::NSLOT];
  __shared__ uint64_t w_bar, done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ float sbias[C::N];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ngroups = (n + C::S - 1) / C::S;
  const int nloc = (int)blockIdx.x < ngroups ? (ngroups - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&in_full[b], LAYER == 1 ? 128 : 1);
      mbar_init(&in_empty[b], 1);
      mbar_init(&st_full[b], 1);
      mbar_init(&st_empty[b], 128);
    }
    for (int i = 0; i < G::NSLOT; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], 128);
    }
    mbar_init(&w_bar, 1);
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < C::N; i += blockDim.x) sbias[i] = bias[i];
  // the buffers' pads are read only for windows nobody keeps; zero them
  for (int i = tid; i < 2 * G::PAD; i += blockDim.x)
    buf0[(i / G::PAD) * G::BUF + C::CB * G::CBS + i % G::PAD] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == WARP_MMA) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tmem_base;
  volatile int* abort = &abort_flag;
#ifdef RBTC_WAIT_PROFILE
  long long ct_acc_[CT_NKIND] = {};
  const long long ct_start_ = clock64();
#endif

  if (warp == WARP_COPY) {
    // ---- copies: the weight image once, then every group's input
    if (lane == 0) {
      mbar_arrive_expect_tx(&w_bar, (unsigned)G::IMG);
      bulk_g2s(bimg, img, (unsigned)G::IMG, &w_bar);
      int k = 0;
      for (; k < nloc; ++k) {
        const int b = k & 1, g = (int)blockIdx.x + k * (int)gridDim.x;
        uint64_t* empty = LAYER == 1 ? &st_empty[b] : &in_empty[b];
        CT_T0();
        const bool ok_e = k < 2 || wait_phase(empty, (unsigned)(((k >> 1) - 1) & 1), abort);
        CT_ACC(CT_COPY_EMPTY);
        if (!ok_e) break;
        issue_group_copy<LAYER>(in, g, n, n_alloc, buf0 + b * G::BUF, stage0 + b * G::STAGE,
                                LAYER == 1 ? &st_full[b] : &in_full[b]);
      }
      // what was issued lands before the shared memory goes
      for (int j = std::max(0, k - 2); j < k; ++j) {
        uint64_t* full = LAYER == 1 ? &st_full[j & 1] : &in_full[j & 1];
        for (int it = 0; it < kMaxSpin && !mbar_try_wait(full, (unsigned)((j >> 1) & 1)); ++it) {
        }
      }
      for (int it = 0; it < kMaxSpin && !mbar_try_wait(&w_bar, 0); ++it) {
      }
    }
  } else if (LAYER == 1 && warp >= WARP_BUILD) {
    // ---- conv1: staged stamps -> input buffer records
    const int t = tid - 32 * WARP_BUILD;
    for (int k = 0; k < nloc; ++k) {
      const int b = k & 1, g = (int)blockIdx.x + k * (int)gridDim.x, ns = min(C::S, n - g * C::S);
      {
        CT_T0();
        const bool ok_s = wait_phase(&st_full[b], (unsigned)((k >> 1) & 1), abort);
        CT_ACC(CT_BUILD_STAGE);
        if (!ok_s) break;
      }
      {
        CT_T0();
        const bool ok_e = k < 2 || wait_phase(&in_empty[b], (unsigned)(((k >> 1) - 1) & 1), abort);
        CT_ACC(CT_BUILD_EMPTY);
        if (!ok_e) break;
      }
      CT_T0();
      build_conv1(ns, buf0 + b * G::BUF, reinterpret_cast<const bf16*>(stage0 + b * G::STAGE), t);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      CT_ACC(CT_BUILD_WORK);
      mbar_arrive(&in_full[b]);
      mbar_arrive(&st_empty[b]);
    }
  } else if (warp == WARP_MMA) {
    // ---- MMAs: per tile, 4 window positions x NTAP taps x KS slices (conv1:
    // 4 row offsets, each over all positions)
    constexpr uint32_t idesc = instr_desc(1, G::NMMA);
    const uint64_t bdesc0 = smem_desc_kn(smem_u32(bimg), 16 * G::NMMA, 128);
    bool live = __all_sync(0xffffffffu, wait_phase(&w_bar, 0, abort));   // warp-uniform: .aligned ops follow
    int tc = 0;
    for (int k = 0; live && k < nloc; ++k) {
      const int b = k & 1;
      {
        CT_T0();
        const bool ok_f = __all_sync(0xffffffffu, wait_phase(&in_full[b], (unsigned)((k >> 1) & 1), abort));
        CT_ACC(CT_MMA_FULL);
        if (!ok_f) break;
      }
      const uint64_t adesc0 = smem_desc_kn(smem_u32(buf0 + b * G::BUF), G::CBS * 16, 128);
      for (int t = 0; t < G::T; ++t, ++tc) {
        const int slot = tc % G::NSLOT;
        {
          CT_T0();
          const unsigned par = (unsigned)((tc / G::NSLOT - 1) & 1);
          const bool ok_a = tc < G::NSLOT || __all_sync(0xffffffffu, wait_phase(&acc_empty[slot], par, abort));
          CT_ACC(CT_MMA_ACC_EMPTY);
          if (!ok_a) {
            live = false;
            break;
          }
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        CT_T0();
        if (lane == 0) {
          if constexpr (LAYER == 1) {
            // one MMA per padded-row offset over all four window positions
            const uint32_t dcol = tbase + (uint32_t)(slot * G::ACC);
#pragma unroll
            for (int ro = 0; ro < 4; ++ro) {
              const int rec = (ro & 1) * G::GW + t * 128 + (ro >> 1) * C::WS;
              mma_bf16(dcol, adesc0 + (uint64_t)rec, bdesc0 + (uint64_t)(ro * 2 * G::NMMA), idesc, ro ? 1u : 0u);
            }
          } else {
#pragma unroll 1
            for (int pos = 0; pos < 4; ++pos) {
              const int a = pos >> 1, bb = pos & 1;
              const uint32_t dcol = tbase + (uint32_t)(slot * G::ACC + pos * C::N);
#pragma unroll
              for (int j = 0; j < C::NTAP; ++j) {
                // padded offsets of the tap: rows a + dy + 1, columns b + dx + 1
                const int ro = a + j / 3, co = bb + j % 3;
                const int rec = ((ro & 1) * 2 + (co & 1)) * G::GW + t * 128 + (ro >> 1) * C::WS + (co >> 1);
#pragma unroll
                for (int ks = 0; ks < G::KS; ++ks) {
                  const uint64_t ad = adesc0 + (uint64_t)(2 * ks * G::CBS + rec);
                  const uint64_t bd = bdesc0 + (uint64_t)((j * G::KS + ks) * 2 * C::N);
                  mma_bf16(dcol, ad, bd, idesc, (j | ks) ? 1u : 0u);
                }
              }
            }
          }
          mma_commit(&acc_full[slot]);
        }
        __syncwarp();
        CT_ACC(CT_MMA_ISSUE);
      }
      if (!live) break;
      if (lane == 0) mma_commit(&in_empty[b]);   // the buffer is free once these MMAs complete
      __syncwarp();
    }
    // every MMA issued completes before the tensor memory is freed
    if (lane == 0) mma_commit(&done_bar);
    __syncwarp();
    for (int it = 0; it < kMaxSpin && !mbar_try_wait(&done_bar, 0); ++it) {
    }
  } else if (warp < 4) {
    // ---- epilogue: thread = window (tensor-memory lane); max over the four
    // window positions, bias, ReLU, BF16 records of the next layer
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    int tc = 0;
    for (int k = 0; k < nloc; ++k) {
      const int g = (int)blockIdx.x + k * (int)gridDim.x, s0 = g * C::S, ns = min(C::S, n - s0);
      bool live = true;
      for (int t = 0; t < G::T; ++t, ++tc) {
        const int slot = tc % G::NSLOT;
        {
          CT_T0();
          const unsigned par = (unsigned)((tc / G::NSLOT) & 1);
          const bool ok_f = __all_sync(0xffffffffu, wait_phase(&acc_full[slot], par, abort));
          CT_ACC(CT_EPI_FULL);
          if (!ok_f) {
            live = false;
            break;
          }
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        CT_T0();
        const int m = t * 128 + 32 * warp + lane, s = m / G::SP, wy = (m % G::SP) / C::WS, wx = m % C::WS;
        const bool keep = s < ns && wy < C::PH && wx < C::PH;
        const uint32_t col0 = tbase + lane_off + (uint32_t)(slot * G::ACC);
#pragma unroll 1
        for (int ch = 0; ch < C::N / 32; ++ch) {
          float u[128], v[32];   // the chunk's 32 channels at the four window positions, one wait
          tmem_ld4x32(col0 + 32 * ch, C::N, u);
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = fmaxf(fmaxf(u[i], u[32 + i]), fmaxf(u[64 + i], u[96 + i]));
          if (keep) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {   // channel block 4 ch + q
              float o[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) o[i] = fmaxf(v[8 * q + i] + sbias[32 * ch + 8 * q + i], 0.f);
              const uint4 rec =
                  make_uint4(pack2(o[0], o[1]), pack2(o[2], o[3]), pack2(o[4], o[5]), pack2(o[6], o[7]));
              const int cbo = 4 * ch + q;
              size_t at;   // record index of the output
              if constexpr (C::NHWC) {
                at = ((size_t)(s0 + s) * 9 + wy * 3 + wx) * 8 + cbo;
              } else {
                const int r = wy + 1, c = wx + 1;   // padded output pixel
                at = ((size_t)(cbo * 4 + (r & 1) * 2 + (c & 1)) * n_alloc + (s0 + s)) * (C::WSO * C::WSO) +
                     (r >> 1) * C::WSO + (c >> 1);
              }
              reinterpret_cast<uint4*>(out)[at] = rec;
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&acc_empty[slot]);
        CT_ACC(CT_EPI_WORK);
      }
      if (!live) break;
    }
  }

  // ---- teardown
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
#ifdef RBTC_WAIT_PROFILE
  if (tid == 0) ct_acc_[CT_CTA] = clock64() - ct_start_;
  if (lane == 0)
    for (int k = 0; k < CT_NKIND; ++k)
      if (ct_acc_[k]) atomicAdd(&g_conv_time[LAYER - 1][k], (unsigned long long)ct_acc_[k]);
#endif
  if (tid == 0 && *abort) atomicOr(err, 1);
  if (warp == WARP_MMA)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
}

// Weight images.  conv2 and conv3: element (j, ks, kc, co, e) sits at
// (((j KS + ks) 2 + kc) N + co) 8 + e and holds the weight of input channel
// (2 ks + kc) 8 + e of tap j.  conv1: element (ro, kc, n, e), n = 32 pos + co,
// sits at ((ro 2 + kc) 128 + n) 8 + e; for window position pos = 2 a + b and
// K entry k = 8 kc + e = 3 px + c (k < 12) it holds the weight of kernel row
// ro - a, column px - b, channel c when both lie in 0 .. 2, else zero.
// Masters in GEMM layout [(tap cin + ci)][cout].
__global__ void k_weight_images(const float* __restrict__ w1, const float* __restrict__ w2,
                                const float* __restrict__ w3, bf16* __restrict__ img1, bf16* __restrict__ img2,
                                bf16* __restrict__ img3) {
  const int total = kWImg1 + kWImg2 + kWImg3;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    int i = idx;
    float v = 0.f;
    bf16* img;
    if (i < kWImg1) {
      img = img1;
      const int e = i & 7, n = (i >> 3) & 127, kc = (i >> 10) & 1, ro = i >> 11;
      const int pos = n >> 5, co = n & 31, a = pos >> 1, b = pos & 1, k = 8 * kc + e;
      const int px = k / 3, c = k % 3, ky = ro - a, kx = px - b;
      if (k < 12 && ky >= 0 && ky < 3 && kx >= 0 && kx < 3) v = w1[((ky * 3 + kx) * 3 + c) * 32 + co];
    } else {
      int N, KS, cin;
      const float* w;
      if ((i -= kWImg1) < kWImg2) {
        N = 64, KS = 2, cin = 32, w = w2, img = img2;
      } else {
        i -= kWImg2;
        N = 64, KS = 4, cin = 64, w = w3, img = img3;
      }
      const int e = i & 7, co = (i >> 3) % N, kc = (i / (8 * N)) & 1, jks = i / (16 * N);
      const int ks = jks % KS, j = jks / KS;
      v = w[(j * cin + (2 * ks + kc) * 8 + e) * N + co];
    }
    img[i] = __float2bfloat16(v);
  }
}

template <int LAYER>
cudaError_t launch(const bf16* in, int n, int n_alloc, const bf16* img, const float* bias, bf16* out, int* err,
                   cudaStream_t s) {
  using G = Geo<LAYER>;
  if (n <= 0) return cudaSuccess;
  static int sms = 0;
  if (sms == 0) {   // one persistent CTA per SM (its shared memory and 512 tensor-memory columns)
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc<LAYER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
  }
  static_assert(2 * (G::SMEM + 2048) > 228 * 1024, "one CTA per SM: each holds all 512 tensor-memory columns");
  const int ngroups = (n + Cfg<LAYER>::S - 1) / Cfg<LAYER>::S;
  k_conv_tc<LAYER><<<std::min(ngroups, sms), 32 * G::NWARP, G::SMEM, s>>>(in, n, n_alloc, img, bias, out, err);
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

extern "C" sfft_status_t rb_debug_conv_waits(int32_t layer, uint64_t* out, int32_t reset) {
#ifdef RBTC_WAIT_PROFILE
  if (!out || layer < 1 || layer > 3) return SFFT_ERR_ARG;
  unsigned long long h[3][rbtc::CT_NKIND];
  if (cudaMemcpyFromSymbol(h, rbtc::g_conv_time, sizeof(h)) != cudaSuccess) return SFFT_ERR_CUDA;
  for (int k = 0; k < rbtc::CT_NKIND; ++k) out[k] = h[layer - 1][k];
  if (reset) {
    const unsigned long long z[rbtc::CT_NKIND] = {};
    if (cudaMemcpyToSymbol(rbtc::g_conv_time, z, sizeof(z), sizeof(z) * (layer - 1)) != cudaSuccess)
      return SFFT_ERR_CUDA;
  }
  return SFFT_OK;
#else
  (void)layer;
  (void)out;
  (void)reset;
  return SFFT_ERR_UNSUPPORTED;
#endif
}
