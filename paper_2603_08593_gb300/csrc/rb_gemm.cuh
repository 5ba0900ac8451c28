// Implicit-GEMM engine of the stamp classifier: C[M][N] = A[M][K] B[K][N] on
// mma.sync m16n8k16 BF16 with FP32 accumulation, 128 x 64 x 32 CTA tiles
// (8 warps of 32 x 32), operands staged through double-buffered shared memory
// in 16-byte vectors and read with ldmatrix.
//
// Operands come from loaders that return 8 consecutive BF16 values along one
// dimension: a "K-major" operand yields (row, k .. k + 7) and is stored as
// [row][k]; an "outer-major" operand yields (k, row .. row + 7) and is stored
// as [k][row], read with ldmatrix.trans.  Loaders hide the convolution
// geometry, so no im2col matrix is ever written:
//   ConvRows   x NHWC [n][h][w][c], row = output pixel, k = (ky * 3 + kx) * c + ci;
//              the source pixel is p + (ky - 1, kx - 1) (forward) or
//              p - (ky - 1, kx - 1) (input gradient); zero outside the image
//   Conv1Rows  the same for c = 3 (k padded to 32), element by element
//   Dense      a row-major matrix [rows][ld]
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace rbg {

using bf16 = __nv_bfloat16;
constexpr int BM = 128, BN = 64, BK = 32, SK = BK + 8;   // SK: padded row of a K-major tile
constexpr int SO_A = BM + 8, SO_B = BN + 8;              // padded rows of outer-major tiles

__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }

// ---------------------------------------------------------------- loaders
struct Dense {
  const bf16* p;
  int rows, cols, ld;   // the matrix is [rows][cols] with row stride ld (a multiple of 8)
  // 8 values along the contiguous dimension: (r, c .. c + 7)
  __device__ __forceinline__ uint4 row8(int r, int c) const {
    if (r >= rows || c >= cols) return zero4();
    return *reinterpret_cast<const uint4*>(p + (int64_t)r * ld + c);
  }
};

struct ConvRows {   // c % 8 == 0
  const bf16* x;
  int n, h, w, c, dir;
  __device__ __forceinline__ uint4 row8(int pix, int k) const {
    if (pix >= n * h * w || k >= 9 * c) return zero4();
    const int tap = k / c, ci = k - tap * c;
    const int xx = pix % w, t = pix / w, yy = t % h, nn = t / h;
    const int sy = yy + dir * (tap / 3 - 1), sx = xx + dir * (tap % 3 - 1);
    if (sy < 0 || sy >= h || sx < 0 || sx >= w) return zero4();
    return *reinterpret_cast<const uint4*>(x + (((int64_t)nn * h + sy) * w + sx) * c + ci);
  }
};

struct Conv1Rows {   // c = 3, k = (ky * 3 + kx) * 3 + ci < 27, padded to 32
  const bf16* x;       // NHWC stamps, sstride values apart
  int n, h, w, sstride;
  __device__ __forceinline__ uint4 row8(int pix, int k) const {
    __align__(16) bf16 v[8];
    const bool okp = pix < n * h * w;
    const int xx = okp ? pix % w : 0, t = okp ? pix / w : 0, yy = t % h, nn = t / h;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int kk = k + j;
      bf16 e = __float2bfloat16(0.f);
      if (okp && kk < 27) {
        const int tap = kk / 3, ci = kk - tap * 3;
        const int sy = yy + tap / 3 - 1, sx = xx + tap % 3 - 1;
        if (sy >= 0 && sy < h && sx >= 0 && sx < w) e = x[(int64_t)nn * sstride + (sy * w + sx) * 3 + ci];
      }
      v[j] = e;
    }
    return *reinterpret_cast<const uint4*>(v);
  }
};

// ---------------------------------------------------------------- fragments
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldm_x4(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldm_x4_t(unsigned (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(smem_addr(p)));
}

__device__ __forceinline__ void mma16816(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ---------------------------------------------------------------- kernel
// A_KM: A is K-major (loader row = m, contiguous k) else outer-major (loader
// row = k, contiguous m).  B_KM: B is K-major (loader row = n, contiguous k)
// else outer-major (loader row = k, contiguous n).  Split K over gridDim.z in
// slices of kchunk (a multiple of BK); slice z writes C + z * cz.
// Epilogue: C[m * ldc + n] (or C[n * ldc + m] with TRANS_C) = acc (+ bias[n]).
template <class LA, class LB, bool A_KM, bool B_KM, bool TRANS_C>
__global__ void __launch_bounds__(256)
k_igemm(int M, int N, int K, int kchunk, LA la, LB lb, float* __restrict__ C, int ldc, int64_t cz,
        const float* __restrict__ bias) {
  constexpr int A_ELEMS = A_KM ? BM * SK : BK * SO_A;
  constexpr int B_ELEMS = B_KM ? BN * SK : BK * SO_B;
  __shared__ __align__(16) bf16 sA[2][A_ELEMS];
  __shared__ __align__(16) bf16 sB[2][B_ELEMS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 3, wn = warp >> 2;   // warp tile rows wm * 32, cols wn * 32
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  C += (int64_t)blockIdx.z * cz;

  // per-thread load slots: A 128 x 32 = 512 vectors (2 per thread), B 64 x 32 = 256 (1 per thread)
  auto load_tile = [&](int k0, uint4 (&ra)[2], uint4& rb) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int v = tid + 256 * j;
      if (A_KM) {   // v -> (m = v / 4, k = (v % 4) * 8)
        const int m = v >> 2, k = k0 + (v & 3) * 8;
        ra[j] = (k < kend) ? la.row8(m0 + m, k) : zero4();
      } else {      // v -> (k = v / 16, m = (v % 16) * 8)
        const int k = k0 + (v >> 4), m = (v & 15) * 8;
        ra[j] = (k < kend) ? la.row8(k, m0 + m) : zero4();
      }
    }
    if (B_KM) {     // tid -> (n = tid / 4, k = (tid % 4) * 8)
      const int n = tid >> 2, k = k0 + (tid & 3) * 8;
      rb = (k < kend) ? lb.row8(n0 + n, k) : zero4();
    } else {        // tid -> (k = tid / 8, n = (tid % 8) * 8)
      const int k = k0 + (tid >> 3), n = (tid & 7) * 8;
      rb = (k < kend) ? lb.row8(k, n0 + n) : zero4();
    }
  };
  auto store_tile = [&](int buf, const uint4 (&ra)[2], const uint4& rb) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int v = tid + 256 * j;
      bf16* dst = A_KM ? &sA[buf][(v >> 2) * SK + (v & 3) * 8] : &sA[buf][(v >> 4) * SO_A + (v & 15) * 8];
      *reinterpret_cast<uint4*>(dst) = ra[j];
    }
    bf16* dst = B_KM ? &sB[buf][(tid >> 2) * SK + (tid & 3) * 8] : &sB[buf][(tid >> 3) * SO_B + (tid & 7) * 8];
    *reinterpret_cast<uint4*>(dst) = rb;
  };

  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  uint4 ra[2], rb;
  int buf = 0;
  if (kbeg < kend) {
    load_tile(kbeg, ra, rb);
    store_tile(0, ra, rb);
  }
  __syncthreads();
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) load_tile(k0 + BK, ra, rb);   // global loads in flight during the MMAs
    const bf16* A = sA[buf];
    const bf16* Bm = sB[buf];
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      unsigned af[2][4], bfr[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm * 32 + i * 16;
        if (A_KM) {   // matrices: (rows 0-7 | 8-15) x (k 0-7 | 8-15)
          ldm_x4(af[i], A + (r + (lane & 7) + ((lane >> 3) & 1) * 8) * SK + kk + (lane >> 4) * 8);
        } else {      // stored [k][m]: transposed 8 x 8 blocks
          ldm_x4_t(af[i], A + (kk + (lane & 7) + (lane >> 4) * 8) * SO_A + r + ((lane >> 3) & 1) * 8);
        }
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {   // 16 columns per ldmatrix.x4: (n 0-7 | 8-15) x (k 0-7 | 8-15)
        const int c = wn * 32 + j * 16;
        if (B_KM) {
          ldm_x4(bfr[j], Bm + (c + (lane & 7) + (lane >> 4) * 8) * SK + kk + ((lane >> 3) & 1) * 8);
        } else {
          ldm_x4_t(bfr[j], Bm + (kk + (lane & 7) + ((lane >> 3) & 1) * 8) * SO_B + c + (lane >> 4) * 8);
        }
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma16816(acc[i][j], af[i], bfr[j >> 1][(j & 1) * 2], bfr[j >> 1][(j & 1) * 2 + 1]);
    }
    if (more) store_tile(buf ^ 1, ra, rb);
    __syncthreads();
    buf ^= 1;
  }
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = m0 + wm * 32 + i * 16 + g, c = n0 + wn * 32 + j * 8 + 2 * t;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int rr = r + (q >= 2 ? 8 : 0), cc = c + (q & 1);
        if (rr < M && cc < N) {
          const float v = acc[i][j][q] + (bias ? bias[cc] : 0.f);
          if (TRANS_C) C[(int64_t)cc * ldc + rr] = v;
          else C[(int64_t)rr * ldc + cc] = v;
        }
      }
    }
}

}  // namespace rbg
