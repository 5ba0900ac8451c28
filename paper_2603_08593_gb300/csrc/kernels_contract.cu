// Lag contraction of row spectra into the normal matrix.
//
// For a probe spectrum P^(y, k) (row FFT of R_m(z) R_m(z + d) for the KK
// block, or of R_m itself for KB and b_K) and weight spectra V^_a(y, k) (row
// FFTs of M_fit xt^a, or of M_fit xt^a S'), the correlation
//   g_{a,b}(u) = sum_x M_fit xt^a yt^b (x) p(x - u)
// is evaluated exactly (circular indexing never wraps because M_fit vanishes
// within w of every edge) in two steps:
//   C_{a,b}(u_y, k) = sum_y yt^b conj(V^_a(y, k)) P^(y - u_y, k)      (y sum, FP32)
//   g_{a,b}(u_y, u_x) = (1/Nf) sum_k h_k Re[C e^{-2 pi i k u_x / Nf}]  (lag DFT)
// with h_0 = h_{Nf/2} = 1, else 2.  The y sum runs over one band of rows per
// CTA with the whole (u_y, monomial) accumulator set of one k-slot held in
// registers; each band ends with the lag DFT over the CTA's k-slots, a warp
// shuffle reduction, a shared-memory reduction over warps and an FP64 global
// atomic add.  Threads own one k-slot and one group of monomials: a group is
// one or two exponents a with all their b (at most five monomials), so one
// complex product conj(V^_a) P^ feeds up to five FMA pairs.
//
// Slot 0 packs the real bins k = 0 and Nf/2 as (re, im); its thread forms the
// two real products instead of a complex product by using per-thread
// coefficients (c1, c2, c3, c4): X = (c1 Pr + c2 Pi, c3 Pi + c4 Pr).
#include "common.cuh"
#include "plan.h"

namespace sfft {

template <int DM, int G> struct GroupCfg { static constexpr int ALO = 0, NLO = 0, AHI = 0, NHI = 0; };
// DM = 4: {a=0: 5}, {a=1: 4, a=4: 1}, {a=2: 3, a=3: 2}
template <> struct GroupCfg<4, 0> { static constexpr int ALO = 0, NLO = 5, AHI = 0, NHI = 0; };
template <> struct GroupCfg<4, 1> { static constexpr int ALO = 1, NLO = 4, AHI = 4, NHI = 1; };
template <> struct GroupCfg<4, 2> { static constexpr int ALO = 2, NLO = 3, AHI = 3, NHI = 2; };
// DM = 3: {a=0: 4}, {a=1: 3, a=3: 1}, {a=2: 2}
template <> struct GroupCfg<3, 0> { static constexpr int ALO = 0, NLO = 4, AHI = 0, NHI = 0; };
template <> struct GroupCfg<3, 1> { static constexpr int ALO = 1, NLO = 3, AHI = 3, NHI = 1; };
template <> struct GroupCfg<3, 2> { static constexpr int ALO = 2, NLO = 2, AHI = 0, NHI = 0; };
// DM = 2: {a=0: 3}, {a=1: 2, a=2: 1}
template <> struct GroupCfg<2, 0> { static constexpr int ALO = 0, NLO = 3, AHI = 0, NHI = 0; };
template <> struct GroupCfg<2, 1> { static constexpr int ALO = 1, NLO = 2, AHI = 2, NHI = 1; };
// DM = 1: {a=0: 2, a=1: 1}
template <> struct GroupCfg<1, 0> { static constexpr int ALO = 0, NLO = 2, AHI = 1, NHI = 1; };
// DM = 0: {a=0: 1}
template <> struct GroupCfg<0, 0> { static constexpr int ALO = 0, NLO = 1, AHI = 0, NHI = 0; };

template <int DM> constexpr int n_groups() { return DM >= 3 ? 3 : (DM == 2 ? 2 : 1); }
template <typename T> constexpr int max_uy() { return sizeof(T) == 4 ? 11 : 6; }

// ---------------------------------------------------------------- shared-memory pipeline
// A CTA walks its band of weight rows y in chunks of CH rows.  For each chunk
// it stages, with cp.async (16-byte copies, double buffered), the probe rows
// z = y - u_y for every lag of the chunk (CH + nuy - 1 rows) and the weight
// rows of every exponent a <= DM, restricted to the CTA's KT k-slots.  The
// arithmetic then reads shared memory only.
constexpr int kChunk = 8;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T, int DM, int KT, int MU>
struct Stage {
  c_t<T> P[kChunk + MU - 1][KT];
  c_t<T> V[DM + 1][kChunk][KT];
};

// issue the copies of chunk [yc, ye) into stage `st`
template <typename T, int DM, int KT, int MU>
__device__ __forceinline__ void stage_chunk(Stage<T, DM, KT, MU>& st, const c_t<T>* __restrict__ P,
                                            const c_t<T>* __restrict__ V, int64_t HM, int M, int k0, int yc, int ye,
                                            int uy_lo, int uy_hi) {
  constexpr int PER_ROW = KT * (int)sizeof(c_t<T>) / 16;   // 16-byte pieces per row segment
  const int np = (ye - yc) + (uy_hi - uy_lo);             // probe rows z = yc - uy_hi ... ye - 1 - uy_lo
  const int nv = (ye - yc);
  const int total = (np + (DM + 1) * nv) * PER_ROW;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int row = t / PER_ROW, piece = t % PER_ROW;
    if (k0 + piece * 16 / (int)sizeof(c_t<T>) >= M) continue;   // k-tile wider than the row (tiny W)
    const c_t<T>* src;
    char* dst;
    if (row < np) {
      const int z = yc - uy_hi + row;
      src = P + (int64_t)z * M + k0;
      dst = reinterpret_cast<char*>(&st.P[row][0]);
    } else {
      const int r2 = row - np, a = r2 / nv, yy = r2 % nv;
      src = V + a * HM + (int64_t)(yc + yy) * M + k0;
      dst = reinterpret_cast<char*>(&st.V[a][yy][0]);
    }
    cp_async16(dst + piece * 16, reinterpret_cast<const char*>(src) + piece * 16);
  }
}

// accumulate the rows [yc, ye) of one staged chunk for monomial group G.
// NUY is the number of lags of the job (compile time, so that the lag loop is
// one straight-line block the scheduler can interleave); NUY = 0 means a
// run-time count `nuy` (used by the FP64 path).
template <typename T, int DM, int KT, int MU, int G, int NUY>
__device__ __forceinline__ void group_chunk(c_t<T> (&acc)[MU][5], const Stage<T, DM, KT, MU>& st, int kk,
                                            bool slot0, int yc, int ye, int nuy_rt, const int* __restrict__ rowflag,
                                            T ysc) {
  using T2 = c_t<T>;
  using C = GroupCfg<DM, G>;
  const int nuy = NUY > 0 ? NUY : nuy_rt;
  for (int y = yc; y < ye; ++y) {
    if (!rowflag[y]) continue;
    const int r = y - yc;
    const T2 vl = st.V[C::ALO][r][kk];
    const T l1 = vl.x, l2 = slot0 ? (T)0 : vl.y, l3 = slot0 ? vl.y : vl.x, l4 = slot0 ? (T)0 : -vl.y;
    T h1 = 0, h2 = 0, h3 = 0, h4 = 0;
    if constexpr (C::NHI > 0) {
      const T2 vh = st.V[C::AHI][r][kk];
      h1 = vh.x; h2 = slot0 ? (T)0 : vh.y; h3 = slot0 ? vh.y : vh.x; h4 = slot0 ? (T)0 : -vh.y;
    }
    const T yt = (T)y * ysc - (T)1;
    T yp[5];
    yp[0] = 1;
#pragma unroll
    for (int b = 1; b < 5; ++b) yp[b] = yp[b - 1] * yt;
    // probe row for lag index iu: z = y - uy_lo - iu  ->  staged row r + (nuy - 1) - iu
    const T2* prow = &st.P[r + nuy - 1][kk];
#pragma unroll
    for (int iu = 0; iu < (NUY > 0 ? NUY : MU); ++iu) {
      if (NUY > 0 || iu < nuy) {
        const T2 pv = prow[-iu * KT];
        const T xr = l1 * pv.x + l2 * pv.y, xi = l3 * pv.y + l4 * pv.x;
#pragma unroll
        for (int s = 0; s < C::NLO; ++s) { acc[iu][s].x += yp[s] * xr; acc[iu][s].y += yp[s] * xi; }
        if constexpr (C::NHI > 0) {
          const T hr = h1 * pv.x + h2 * pv.y, hi = h3 * pv.y + h4 * pv.x;
#pragma unroll
          for (int s = 0; s < C::NHI; ++s) { acc[iu][C::NLO + s].x += yp[s] * hr; acc[iu][C::NLO + s].y += yp[s] * hi; }
        }
      }
    }
  }
}

// lag DFT over this thread's k, warp reduction over 32 k-slots, shared accumulation
template <typename T, int DM, int MU, int G>
__device__ __forceinline__ void group_flush(const c_t<T> (&acc)[MU][5], const CJob& job, int k, int Nf, int L,
                                            T* red, const c_t<T>* __restrict__ twD) {
  using T2 = c_t<T>;
  using C = GroupCfg<DM, G>;
  constexpr int NS = C::NLO + C::NHI;
  constexpr int NMONO = n_mono(DM);
  const int lane = threadIdx.x & 31;
  const int nuy = job.uy_hi - job.uy_lo + 1;
  const int w = (L - 1) / 2;
  const bool slot0 = (k == 0);
  for (int ux = job.ux_lo; ux <= job.ux_hi; ++ux) {
    T tre, tim;
    if (slot0) {
      tre = 1; tim = (ux & 1) ? (T)-1 : (T)1;
    } else {
      int idx = (int)(((int64_t)k * ux) % Nf);
      if (idx < 0) idx += Nf;
      const T2 cs = twD[idx];
      tre = 2 * cs.x; tim = 2 * cs.y;
    }
#pragma unroll
    for (int iu = 0; iu < MU; ++iu) {
      if (iu < nuy) {
        const int ridx = ((job.uy_lo + iu + w) * L + (ux + w)) * NMONO;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          T v = acc[iu][s].x * tre + acc[iu][s].y * tim;
          v = warp_sum(v);
          if (lane == 0) {
            const int m = s < C::NLO ? mono_index(C::ALO, s) : mono_index(C::AHI, s - C::NLO);
            atomicAdd(&red[ridx + m], v);
          }
        }
      }
    }
  }
}

template <typename T, int DM, int KT>
__global__ void __launch_bounds__(KT * n_groups<DM>(), 1)
k_contract(const CJob* __restrict__ jobs, char* __restrict__ ws, int H, int M, int Nf, int L, int rows_per_cta,
           const c_t<T>* __restrict__ twD) {
  using T2 = c_t<T>;
  constexpr int MU = max_uy<T>();
  constexpr int NMONO = n_mono(DM);
  using St = Stage<T, DM, KT, MU>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  St* stages = reinterpret_cast<St*>(smem_raw);
  T* red = reinterpret_cast<T*>(smem_raw + 2 * sizeof(St));   // [L][L][n_mono(DM)]
  const CJob job = jobs[blockIdx.z];
  const int nred = L * L * NMONO;
  for (int i = threadIdx.x; i < nred; i += blockDim.x) red[i] = (T)0;

  const int w = (L - 1) / 2;
  const int g = threadIdx.x / KT, kk = threadIdx.x % KT;
  const int k0 = blockIdx.x * KT, k = k0 + kk;
  int y0 = blockIdx.y * rows_per_cta, y1 = y0 + rows_per_cta;
  if (y0 < w) y0 = w;
  if (y1 > H - w) y1 = H - w;
  const int64_t HM = (int64_t)H * M;
  const T2* P = reinterpret_cast<const T2*>(ws + job.probe);
  const T2* V = reinterpret_cast<const T2*>(ws + job.wts);
  const int* rowflag = reinterpret_cast<const int*>(ws + job.rowflag);
  const int nuy = job.uy_hi - job.uy_lo + 1;
  const T ysc = (T)2 / (T)(H > 1 ? H - 1 : 1);
  const bool slot0 = (k == 0);

  T2 acc[MU][5];
#pragma unroll
  for (int i = 0; i < MU; ++i)
#pragma unroll
    for (int s = 0; s < 5; ++s) { acc[i][s].x = 0; acc[i][s].y = 0; }

  const int nchunk = y1 > y0 ? (y1 - y0 + kChunk - 1) / kChunk : 0;
  if (nchunk > 0) {
    stage_chunk<T, DM, KT, MU>(stages[0], P, V, HM, M, k0, y0, min(y0 + kChunk, y1), job.uy_lo, job.uy_hi);
    cp_async_commit();
  }
  for (int c = 0; c < nchunk; ++c) {
    const int yc = y0 + c * kChunk, ye = min(yc + kChunk, y1);
    if (c + 1 < nchunk) {
      const int yn = yc + kChunk;
      stage_chunk<T, DM, KT, MU>(stages[(c + 1) & 1], P, V, HM, M, k0, yn, min(yn + kChunk, y1), job.uy_lo,
                                 job.uy_hi);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const St& st = stages[c & 1];
    if constexpr (sizeof(T) == 4) {
      switch (nuy) {
#define SFFT_NUY_CASE(NV)                                                                                      \
  case NV:                                                                                                     \
    if (g == 0) group_chunk<T, DM, KT, MU, 0, NV>(acc, st, kk, slot0, yc, ye, nuy, rowflag, ysc);              \
    if constexpr (n_groups<DM>() > 1) {                                                                        \
      if (g == 1) group_chunk<T, DM, KT, MU, 1, NV>(acc, st, kk, slot0, yc, ye, nuy, rowflag, ysc);            \
    }                                                                                                          \
    if constexpr (n_groups<DM>() > 2) {                                                                        \
      if (g == 2) group_chunk<T, DM, KT, MU, 2, NV>(acc, st, kk, slot0, yc, ye, nuy, rowflag, ysc);            \
    }                                                                                                          \
    break;
        SFFT_NUY_CASE(1) SFFT_NUY_CASE(2) SFFT_NUY_CASE(3) SFFT_NUY_CASE(4) SFFT_NUY_CASE(5) SFFT_NUY_CASE(6)
        SFFT_NUY_CASE(7) SFFT_NUY_CASE(8) SFFT_NUY_CASE(9) SFFT_NUY_CASE(10) SFFT_NUY_CASE(11)
#undef SFFT_NUY_CASE
        default: break;
      }
    } else {
      if (g == 0) group_chunk<T, DM, KT, MU, 0, 0>(acc, st, kk, slot0, yc, ye, nuy, rowflag, ysc);
      if constexpr (n_groups<DM>() > 1) { if (g == 1) group_chunk<T, DM, KT, MU, 1, 0>(acc, st, kk, slot0, yc, ye, nuy, rowflag, ysc); }
      if constexpr (n_groups<DM>() > 2) { if (g == 2) group_chunk<T, DM, KT, MU, 2, 0>(acc, st, kk, slot0, yc, ye, nuy, rowflag, ysc); }
    }
    __syncthreads();
  }
  // k-slots past the row (whole warps, since M and KT are multiples of 32) hold junk
  if (k < M) {
    if (g == 0) group_flush<T, DM, MU, 0>(acc, job, k, Nf, L, red, twD);
    if constexpr (n_groups<DM>() > 1) { if (g == 1) group_flush<T, DM, MU, 1>(acc, job, k, Nf, L, red, twD); }
    if constexpr (n_groups<DM>() > 2) { if (g == 2) group_flush<T, DM, MU, 2>(acc, job, k, Nf, L, red, twD); }
  }
  __syncthreads();
  const double inv = 1.0 / (double)Nf;
  const int nux = job.ux_hi - job.ux_lo + 1;
  const int nval = nuy * nux * NMONO;
  for (int i = threadIdx.x; i < nval; i += blockDim.x) {
    const int m = i % NMONO, t = i / NMONO;
    const int ux = job.ux_lo + t % nux, uy = job.uy_lo + t / nux;
    const int ridx = ((uy + w) * L + (ux + w)) * NMONO + m;
    const T v = red[ridx];
    if (v != (T)0) atomicAdd(reinterpret_cast<double*>(ws + job.out) + ridx, (double)v * inv);
  }
}

template <typename T, int DM, int KT>
static cudaError_t contract_launch(const sfft_plan_s* p, int job0, int njobs, int rows_per_cta, void* ws) {
  const int H = p->d.H, L = p->d.L;
  constexpr int MU = max_uy<T>();
  const size_t smem = 2 * sizeof(Stage<T, DM, KT, MU>) + sizeof(T) * L * L * n_mono(DM);
  auto kern = k_contract<T, DM, KT>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int nb = (H + rows_per_cta - 1) / rows_per_cta;
  dim3 grid((p->M + KT - 1) / KT, nb, njobs);
  kern<<<grid, KT * n_groups<DM>(), smem, p->stream>>>(p->d_jobs + job0, (char*)ws, H, p->M, p->Nf, L, rows_per_cta,
                                                       (const c_t<T>*)p->twD);
  p->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T, int DM>
static cudaError_t contract_T(const sfft_plan_s* p, int job0, int njobs, int rows_per_cta, int ktile, void* ws) {
  // shared memory per stage grows with KT; FP64 stages hold twice the bytes, so FP64 uses KT = 64
  if (sizeof(T) == 8 || ktile == 64) return contract_launch<T, DM, 64>(p, job0, njobs, rows_per_cta, ws);
  return contract_launch<T, DM, 128>(p, job0, njobs, rows_per_cta, ws);
}

template <typename T>
static cudaError_t contract_dm(const sfft_plan_s* p, int DM, int job0, int njobs, int rows_per_cta, int ktile,
                               void* ws) {
  switch (DM) {
    case 0: return contract_T<T, 0>(p, job0, njobs, rows_per_cta, ktile, ws);
    case 1: return contract_T<T, 1>(p, job0, njobs, rows_per_cta, ktile, ws);
    case 2: return contract_T<T, 2>(p, job0, njobs, rows_per_cta, ktile, ws);
    case 3: return contract_T<T, 3>(p, job0, njobs, rows_per_cta, ktile, ws);
    case 4: return contract_T<T, 4>(p, job0, njobs, rows_per_cta, ktile, ws);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_contract(const sfft_plan_s* p, int DM, int job0, int njobs, int rows_per_cta, int ktile,
                            void* ws) {
  if (njobs <= 0) return cudaSuccess;
  return p->fp64 ? contract_dm<double>(p, DM, job0, njobs, rows_per_cta, ktile, ws)
                 : contract_dm<float>(p, DM, job0, njobs, rows_per_cta, ktile, ws);
}

}  // namespace sfft
