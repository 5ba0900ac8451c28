// Helpers shared by the tcgen05 contraction kernels: shared-memory matrix
// and instruction descriptors, tensor-map copies, operand splitting and
// bounded mbarrier waits.
#pragma once
#include <cuda.h>

#include "bulk.cuh"
#include "common.cuh"

namespace sfft {

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo = 256u) {
  // canonical K-major layout without swizzle: core matrices of 8 rows x 16
  // bytes, 128 bytes apart along K (leading byte offset) and `sbo` bytes
  // apart along the 8-row groups (stride byte offset); descriptor version 1
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// canonical K-major layout without swizzle with both strides given: core
// matrices (8 rows x 16 bytes) `lbo` bytes apart along K and `sbo` bytes
// apart along the 8-row groups; descriptor version 1
__device__ __forceinline__ uint64_t smem_desc_kn(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor: D FP32, A and B of format `fmt` (1 = BF16 for
// kind::f16, 2 = TF32 for kind::tf32), both K-major, M = 128, N columns
// (a multiple of 16 up to 256; 32 by default)
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t n = 32) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

// tiled tensor copy of a 3-D box (x innermost) into shared memory, counted on `bar`
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// tiled tensor copy of a 4-D box (x innermost) into shared memory, counted on `bar`
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int v,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(v), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool elect_one() {
  uint32_t pred = 0;
  asm volatile("{\n .reg .pred P;\n elect.sync _|P, 0xffffffff;\n selp.u32 %0, 1, 0, P;\n}\n" : "=r"(pred));
  return pred != 0;
}

__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void mono_ab(int m, int& a, int& b) {
  int n = 0;
  while ((n + 1) * (n + 2) / 2 <= m) ++n;
  b = m - n * (n + 1) / 2;
  a = n - b;
}

// Bounded wait on a phase; gives up when the spin budget runs out or another
// role has given up, and then raises the shared abort flag.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, unsigned parity, volatile int* abort) {
  for (int it = 0; it < kMaxSpin; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 63 && *abort) return false;
  }
  *abort = 1;
  return false;
}


using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
  }
  return fn;
}

// 3-D FP32 view (x: 2 M floats of one spectrum row, y: rows, z: spectra) of
// `n` consecutive row spectra, with boxes of bx floats x by rows x bz spectra
inline bool make_map(CUtensorMap* m, void* base, int M, int H, int n, int bx, int by, int bz) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * M, (cuuint64_t)H, (cuuint64_t)n};
  const cuuint64_t strides[2] = {(cuuint64_t)2 * M * 4, (cuuint64_t)H * 2 * M * 4};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}


// 4-D FP32 view of k-slot-blocked spectra [n][M / 16][H][16 complex] (x: the
// 32 floats of one block row, y: rows, z: blocks, v: spectra), with boxes of
// bx floats x by rows x 1 block x bv spectra
inline bool make_map_blk(CUtensorMap* m, void* base, int M, int H, int n, int bx, int by, int bv) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[4] = {32, (cuuint64_t)H, (cuuint64_t)(M / 16), (cuuint64_t)n};
  const cuuint64_t strides[3] = {128, (cuuint64_t)H * 128, (cuuint64_t)H * 128 * (M / 16)};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, (cuuint32_t)bv};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

}  // namespace sfft
