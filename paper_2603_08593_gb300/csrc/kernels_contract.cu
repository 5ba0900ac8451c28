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
// CTA with the accumulators in registers; each band ends with the lag DFT
// over the CTA's k-slots, a warp shuffle reduction, a shared-memory reduction
// over warps and an FP64 global atomic add.
//
// Thread layout: one k-slot x one monomial group x one part of the lags.  A
// monomial group is one or two exponents a with all their b (at most five
// monomials), so one complex product conj(V^_a) P^ feeds up to five FMA
// pairs; splitting the lags over two threads halves the accumulators per
// thread (at most 6 lags x 5 monomials) so that two or three CTAs fit on an SM.
//
// Slot 0 packs the real bins k = 0 and Nf/2 as (re, im).  The main kernel
// treats it as an ordinary complex slot and drops it at the flush; the small
// kernel k_contract_slot0 adds the two real-bin terms exactly, which keeps the
// hot loop free of per-slot special cases.
#include "bulk.cuh"
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
// NS threads share the lags of one (k, group): lags [p ceil(nuy / NS), ...) go to part p
template <typename T, int NS> constexpr int max_part() { return (max_uy<T>() + NS - 1) / NS; }
__device__ __forceinline__ void lag_part(int nuy, int ns, int part, int& lag0, int& nlag) {
  const int per = (nuy + ns - 1) / ns;
  lag0 = part * per;
  nlag = max(0, min(per, nuy - lag0));
}
// k-slots per CTA: the five-monomial groups (DM >= 3) use 32-slot tiles so
// that three CTAs fit on an SM; FP64 accumulators take one CTA per SM.
template <typename T, int DM> constexpr int kt_for() { return DM >= 3 ? 32 : 64; }
// register cap per thread: three CTAs of 192 threads (DM >= 3, two lag parts) or of 288
// threads (three parts), two CTAs of 256 or 384 threads otherwise, fit in 64K registers
template <typename T, int DM, int NS> constexpr int maxreg_for() {
  return sizeof(T) == 8 ? 255 : (NS == 1 ? 168 : (DM >= 3 ? (NS == 2 ? 96 : 72) : (NS == 2 ? 112 : 80)));
}

// ---------------------------------------------------------------- shared-memory pipeline
// A CTA walks its band of weight rows y in chunks of kChunk rows.  For each
// chunk it stages, with bulk (TMA-engine) copies into two alternating stages,
// the probe rows z = y - u_y for every lag of the chunk (kChunk + nuy - 1
// rows), the weight rows of every exponent a <= DM (restricted to the CTA's
// k-slots), the powers of yt and the row flags.  The chunk after next is in
// flight while a chunk is being consumed; the arithmetic reads shared memory only.
constexpr int kChunk = 16;

template <typename T, int DM, int KT, int MU>
struct Stage {
  c_t<T> P[kChunk + MU - 1][KT];
  c_t<T> V[DM + 1][kChunk][KT];
  T ypw[kChunk][64 / sizeof(T)];   // yt^b of the chunk's rows, b = 0..4, in the power table's 64 B rows
  int rf[kChunk + 4];      // row flags from the 16-byte aligned row at or below the chunk start
};

// Issue the bulk copies of chunk [yc, ye) into stage `st`: one per probe /
// weight row segment of KT slots, one for the powers of yt and one for the row
// flags, each from its own thread, counted on `full`.  Thread 0 registers the
// expected bytes with its arrival; the phase completes once every byte landed.
template <typename T, int DM, int KT, int MU>
__device__ __forceinline__ void produce_chunk(Stage<T, DM, KT, MU>& st, uint64_t* full, const c_t<T>* __restrict__ P,
                                              const c_t<T>* __restrict__ V, const T* __restrict__ ytab,
                                              const int* __restrict__ rowflag, int64_t HM, int M, int k0, int yc,
                                              int ye, int uy_lo, int uy_hi) {
  const int np = (ye - yc) + (uy_hi - uy_lo);             // probe rows z = yc - uy_hi ... ye - 1 - uy_lo
  const int nv = (ye - yc);
  const int slots = min(KT, M - k0);                       // a tile wider than a tiny row copies less
  const unsigned seg = (unsigned)(slots * sizeof(c_t<T>)); // multiple of 256 bytes
  const unsigned ybytes = (unsigned)(nv * 64);
  const unsigned fbytes = (unsigned)((kChunk + 4) * sizeof(int));
  const int ncopy = np + (DM + 1) * nv;
  if (threadIdx.x == 0) mbar_arrive_expect_tx(full, seg * (unsigned)ncopy + ybytes + fbytes);
  // every copy registered above is issued, whatever the CTA size
  for (int t = threadIdx.x; t < ncopy + 2; t += blockDim.x) {
    if (t < np) {
      bulk_copy_g2s(&st.P[t][0], P + (int64_t)(yc - uy_hi + t) * M + k0, seg, full);
    } else if (t < ncopy) {
      const int r2 = t - np, a = r2 / nv, yy = r2 - a * nv;
      bulk_copy_g2s(&st.V[a][yy][0], V + a * HM + (int64_t)(yc + yy) * M + k0, seg, full);
    } else if (t == ncopy) {
      bulk_copy_g2s(&st.ypw[0][0], ytab + (int64_t)yc * (64 / sizeof(T)), ybytes, full);
    } else {
      bulk_copy_g2s(&st.rf[0], rowflag + (yc & ~3), fbytes, full);
    }
  }
}

// Accumulate the rows [yc, ye) of one staged chunk for monomial group G and
// lags iu = lag0 .. lag0 + nlag - 1 (accumulator index iu - lag0).  NLAG > 0
// fixes the lag count at compile time (one straight-line lag block the
// scheduler can interleave); NLAG = 0 uses the run-time count (FP64 path).
// Every slot is treated as a complex bin here, slot 0 included; slot 0 (the
// packed real bins k = 0 and Nf/2) is dropped at the flush and summed exactly
// by k_contract_slot0.
template <typename T, int DM, int KT, int MU, int MH, int G, int NLAG>
__device__ __forceinline__ void group_chunk(c_t<T> (&acc)[MH][5], const Stage<T, DM, KT, MU>& st, int kk,
                                            int nrow, int nuy, int lag0, int nlag_rt, const int* rf) {
  using T2 = c_t<T>;
  using C = GroupCfg<DM, G>;
  const int nlag = NLAG > 0 ? NLAG : nlag_rt;
  for (int r = 0; r < nrow; ++r) {
    if (!rf[r]) continue;   // no fit pixel on this row: its weight spectra are zero
    const T2 vl = st.V[C::ALO][r][kk];
    T2 vh;
    if constexpr (C::NHI > 0) vh = st.V[C::AHI][r][kk];
    T yp[5];
#pragma unroll
    for (int b = 0; b < 5; ++b) yp[b] = st.ypw[r][b];
    // probe row for lag iu: z = y - uy_lo - iu  ->  staged row r + (nuy - 1) - iu
    const T2* prow = &st.P[r + nuy - 1 - lag0][kk];
#pragma unroll
    for (int i = 0; i < (NLAG > 0 ? NLAG : MH); ++i) {
      if (NLAG > 0 || i < nlag) {
        const T2 pv = prow[-i * KT];
        // conj(V) P
        const T xr = vl.x * pv.x + vl.y * pv.y, xi = vl.x * pv.y - vl.y * pv.x;
#pragma unroll
        for (int s = 0; s < C::NLO; ++s) { acc[i][s].x += yp[s] * xr; acc[i][s].y += yp[s] * xi; }
        if constexpr (C::NHI > 0) {
          const T hr = vh.x * pv.x + vh.y * pv.y, hi = vh.x * pv.y - vh.y * pv.x;
#pragma unroll
          for (int s = 0; s < C::NHI; ++s) { acc[i][C::NLO + s].x += yp[s] * hr; acc[i][C::NLO + s].y += yp[s] * hi; }
        }
      }
    }
  }
}

// FP32 hot loop with explicit 32-bit shared-memory addresses: three row
// pointers advance by a constant per row and every load uses a compile-time
// immediate offset, so address arithmetic costs a few integer adds per row.
template <int OFF>
__device__ __forceinline__ float2 lds2(unsigned addr) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(addr), "n"(OFF));
  return v;
}
__device__ __forceinline__ float4 lds4(unsigned addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
  return v;
}

template <int NLAG, int KT, int I>
__device__ __forceinline__ float2 lag_load(unsigned p_lo) {
  // lag i lives (NLAG - 1 - i) staged rows above the lowest row of this thread's lags
  return lds2<(NLAG - 1 - I) * KT * 8>(p_lo);
}

template <int NLAG, int KT, int I>
__device__ __forceinline__ void load_lags(float2 (&pv)[NLAG], unsigned plo) {
  if constexpr (I < NLAG) {
    pv[I] = lag_load<NLAG, KT, I>(plo);
    load_lags<NLAG, KT, I + 1>(pv, plo);
  }
}

template <int DM, int KT, int MU, int MH, int G, int NLAG>
__device__ __forceinline__ void group_chunk_f32(c_t<float> (&acc)[MH][5], const Stage<float, DM, KT, MU>& st, int kk,
                                                int nrow, int nuy, int lag0, const int* rf) {
  using C = GroupCfg<DM, G>;
  unsigned vlo = (unsigned)__cvta_generic_to_shared(&st.V[C::ALO][0][kk]);
  unsigned vhi = (unsigned)__cvta_generic_to_shared(&st.V[C::NHI > 0 ? C::AHI : C::ALO][0][kk]);
  unsigned ypa = (unsigned)__cvta_generic_to_shared(&st.ypw[0][0]);
  // staged row of lag lag0 + NLAG - 1 for r = 0
  unsigned plo = (unsigned)__cvta_generic_to_shared(&st.P[nuy - 1 - lag0 - (NLAG - 1)][kk]);
  for (int r = 0; r < nrow; ++r, vlo += KT * 8, vhi += KT * 8, ypa += 64, plo += KT * 8) {
    if (!rf[r]) continue;   // no fit pixel on this row: its weight spectra are zero
    const float2 vl = lds2<0>(vlo);
    float2 vh = vl;
    if constexpr (C::NHI > 0) vh = lds2<0>(vhi);
    // the powers of yt arrive as duplicated pairs: operands of the packed FMA as loaded
    const float4 y01 = lds4(ypa), y23 = lds4(ypa + 16);
    const float2 yp[5] = {make_float2(y01.x, y01.y), make_float2(y01.z, y01.w), make_float2(y23.x, y23.y),
                          make_float2(y23.z, y23.w), lds2<32>(ypa)};
    const float2 vlx = make_float2(vl.x, vl.x), vhx = make_float2(vh.x, vh.x);
    float2 pv[NLAG];
    load_lags<NLAG, KT, 0>(pv, plo);
#pragma unroll
    for (int i = 0; i < NLAG; ++i) {
      // conj(V) P = (vx px + vy py, vx py - vy px): one packed product and two FMAs
      float2 x = __fmul2_rn(vlx, pv[i]);
      x.x = fmaf(vl.y, pv[i].y, x.x);
      x.y = fmaf(-vl.y, pv[i].x, x.y);
#pragma unroll
      for (int s = 0; s < C::NLO; ++s) acc[i][s] = __ffma2_rn(yp[s], x, acc[i][s]);
      if constexpr (C::NHI > 0) {
        float2 h = __fmul2_rn(vhx, pv[i]);
        h.x = fmaf(vh.y, pv[i].y, h.x);
        h.y = fmaf(-vh.y, pv[i].x, h.y);
#pragma unroll
        for (int s = 0; s < C::NHI; ++s) acc[i][C::NLO + s] = __ffma2_rn(yp[s], h, acc[i][C::NLO + s]);
      }
    }
  }
}

// lag DFT over this thread's k, warp reduction over 32 k-slots, shared accumulation
template <typename T, int DM, int MH, int G>
__device__ __forceinline__ void group_flush(const c_t<T> (&acc)[MH][5], const CJob& job, int k, int Nf, int L,
                                            int lag0, int nlag, T* red, const c_t<T>* __restrict__ twD) {
  using T2 = c_t<T>;
  using C = GroupCfg<DM, G>;
  constexpr int NS = C::NLO + C::NHI;
  constexpr int NMONO = n_mono(DM);
  const int lane = threadIdx.x & 31;
  const int w = (L - 1) / 2;
  const bool slot0 = (k == 0);
  for (int ux = job.ux_lo; ux <= job.ux_hi; ++ux) {
    T tre, tim;
    if (slot0) {
      tre = 0; tim = 0;   // packed real bins: summed by k_contract_slot0
    } else {
      int idx = (int)(((int64_t)k * ux) % Nf);
      if (idx < 0) idx += Nf;
      const T2 cs = twD[idx];
      tre = 2 * cs.x; tim = 2 * cs.y;
    }
#pragma unroll
    for (int i = 0; i < MH; ++i) {
      if (i < nlag) {
        const int ridx = ((job.uy_lo + lag0 + i + w) * L + (ux + w)) * NMONO;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          T v = acc[i][s].x * tre + acc[i][s].y * tim;
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

template <typename T, int DM, int KT, int MU, int MH, int G>
__device__ __forceinline__ void chunk_dispatch(c_t<T> (&acc)[MH][5], const Stage<T, DM, KT, MU>& st, int kk,
                                               int nrow, int nuy, int lag0, int nlag, const int* rf) {
  if constexpr (sizeof(T) == 4) {
    switch (nlag) {
#define SFFT_NLAG_CASE(NV) \
  case NV: group_chunk_f32<DM, KT, MU, MH, G, NV>(acc, st, kk, nrow, nuy, lag0, rf); break;
      SFFT_NLAG_CASE(1) SFFT_NLAG_CASE(2) SFFT_NLAG_CASE(3) SFFT_NLAG_CASE(4) SFFT_NLAG_CASE(5) SFFT_NLAG_CASE(6)
      default: break;
    }
    if constexpr (MH > 6) {   // one lag part: up to 11 lags per thread
      switch (nlag) {
        SFFT_NLAG_CASE(7) SFFT_NLAG_CASE(8) SFFT_NLAG_CASE(9) SFFT_NLAG_CASE(10) SFFT_NLAG_CASE(11)
        default: break;
      }
    }
#undef SFFT_NLAG_CASE
  } else {
    if (nlag > 0) group_chunk<T, DM, KT, MU, MH, G, 0>(acc, st, kk, nrow, nuy, lag0, nlag, rf);
  }
}

template <typename T, int DM, int KT, int NS> constexpr int cta_threads() { return KT * n_groups<DM>() * NS; }

template <typename T, int DM, int KT, int NS>
__global__ void __launch_bounds__(cta_threads<T, DM, KT, NS>()) __maxnreg__((maxreg_for<T, DM, NS>()))
k_contract(const CJob* __restrict__ jobs, char* __restrict__ ws, int H, int M, int Nf, int L, int rows_per_cta,
           const c_t<T>* __restrict__ twD, const T* __restrict__ ytab) {
  using T2 = c_t<T>;
  constexpr int MU = max_uy<T>();
  constexpr int MH = max_part<T, NS>();
  constexpr int NMONO = n_mono(DM);
  constexpr int NG = n_groups<DM>();
  using St = Stage<T, DM, KT, MU>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  St* stages = reinterpret_cast<St*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + 2 * sizeof(St));    // [2]
  T* red = reinterpret_cast<T*>(smem_raw + 2 * sizeof(St) + 32);              // [L][L][n_mono(DM)]
  const CJob job = jobs[blockIdx.y];
  const int nred = L * L * NMONO;
  for (int i = threadIdx.x; i < nred; i += blockDim.x) red[i] = (T)0;
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int w = (L - 1) / 2;
  const int kk = threadIdx.x % KT, gp = threadIdx.x / KT;     // gp = group * NS + part (warp-uniform)
  const int g = gp / NS, part = gp % NS;
  const int k0 = blockIdx.x * KT, k = k0 + kk;
  int y0 = blockIdx.z * rows_per_cta, y1 = y0 + rows_per_cta;
  if (y0 < w) y0 = w;
  if (y1 > H - w) y1 = H - w;
  const int64_t HM = (int64_t)H * M;
  const T2* P = reinterpret_cast<const T2*>(ws + job.probe);
  const T2* V = reinterpret_cast<const T2*>(ws + job.wts);
  const int* rowflag = reinterpret_cast<const int*>(ws + job.rowflag);
  const int nuy = job.uy_hi - job.uy_lo + 1;
  int lag0, nlag;
  lag_part(nuy, NS, part, lag0, nlag);

  T2 acc[MH][5];
#pragma unroll
  for (int i = 0; i < MH; ++i)
#pragma unroll
    for (int s = 0; s < 5; ++s) { acc[i][s].x = 0; acc[i][s].y = 0; }

  const int nchunk = y1 > y0 ? (y1 - y0 + kChunk - 1) / kChunk : 0;
  if (nchunk > 0)
    produce_chunk<T, DM, KT, MU>(stages[0], &full[0], P, V, ytab, rowflag, HM, M, k0, y0, min(y0 + kChunk, y1),
                                 job.uy_lo, job.uy_hi);
  for (int c = 0; c < nchunk; ++c) {
    const int yc = y0 + c * kChunk, ye = min(yc + kChunk, y1);
    if (c + 1 < nchunk) {   // stage (c+1)&1 was released by the barrier that closed chunk c - 1
      const int yn = yc + kChunk;
      produce_chunk<T, DM, KT, MU>(stages[(c + 1) & 1], &full[(c + 1) & 1], P, V, ytab, rowflag, HM, M, k0, yn,
                                   min(yn + kChunk, y1), job.uy_lo, job.uy_hi);
    }
    // stage c & 1 serves chunks c, c + 2, ...: its (c >> 1)-th phase completes chunk c
    const bool landed = mbar_wait_bounded(&full[c & 1], (unsigned)((c >> 1) & 1));
    if (!__syncthreads_and(landed)) {
      // copies never completed: flag the CCD, give the in-flight copies a bounded
      // chance to drain, and leave without touching the accumulators
      if (threadIdx.x == 0) atomicOr(reinterpret_cast<int*>(ws + job.status), 4);
      if (c + 1 < nchunk) mbar_wait_bounded(&full[(c + 1) & 1], (unsigned)(((c + 1) >> 1) & 1));
      return;
    }
    const St& st = stages[c & 1];
    const int* rf = st.rf + (yc & 3);
    if (g == 0) chunk_dispatch<T, DM, KT, MU, MH, 0>(acc, st, kk, ye - yc, nuy, lag0, nlag, rf);
    if constexpr (NG > 1) { if (g == 1) chunk_dispatch<T, DM, KT, MU, MH, 1>(acc, st, kk, ye - yc, nuy, lag0, nlag, rf); }
    if constexpr (NG > 2) { if (g == 2) chunk_dispatch<T, DM, KT, MU, MH, 2>(acc, st, kk, ye - yc, nuy, lag0, nlag, rf); }
    __syncthreads();
  }
  // k-slots past the row (whole warps, since M and KT are multiples of 32) hold junk
  if (k < M) {
    if (g == 0) group_flush<T, DM, MH, 0>(acc, job, k, Nf, L, lag0, nlag, red, twD);
    if constexpr (NG > 1) { if (g == 1) group_flush<T, DM, MH, 1>(acc, job, k, Nf, L, lag0, nlag, red, twD); }
    if constexpr (NG > 2) { if (g == 2) group_flush<T, DM, MH, 2>(acc, job, k, Nf, L, lag0, nlag, red, twD); }
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

// The two real bins packed in slot 0 (k = 0 and k = Nf/2, each with h = 1):
//   g_{a,b}(u) += (1/Nf) sum_y yt^b [V_a(y,0) P(y-u_y,0) + (-1)^{u_x} V_a(y,Nf/2) P(y-u_y,Nf/2)]
// One CTA per (job, band of at most slot0_rows rows y).  The band's slot-0
// values (probe rows y - u_y for every u_y of the job, weight rows y for
// every exponent, row flags) are staged in shared memory once, so each
// scattered 8- or 16-byte value is read from L2 once per band rather than
// once per u_y.  Warp i takes u_y = uy_lo + i and lane l the rows
// y = yb + l (mod 32): per-lane sums and the warp tree in T (FP32 on the
// mixed path), FP64 atomic adds.
template <typename T> constexpr int slot0_rows() { return sizeof(T) == 4 ? 512 : 256; }

template <typename T, int DM>
__global__ void __launch_bounds__(32 * max_uy<T>())
k_contract_slot0(const CJob* __restrict__ jobs, char* __restrict__ ws, int H, int M, int Nf, int L, int rs,
                 int rows_per_band) {
  using T2 = c_t<T>;
  constexpr int NMONO = n_mono(DM), MU = max_uy<T>(), RB = slot0_rows<T>();
  __shared__ T2 ps[RB + MU - 1];
  __shared__ T2 vs[DM + 1][RB];
  __shared__ int fl[RB];
  __shared__ double red[MU][2 * NMONO];
  const CJob job = jobs[blockIdx.x];
  const int nuy = job.uy_hi - job.uy_lo + 1;   // at most MU (jobs are split by u_y)
  const int w = (L - 1) / 2;
  const int yb = w + (int)blockIdx.y * rows_per_band, ye = min(H - w, yb + rows_per_band);
  const int nr = ye - yb;                      // at most RB
  const int64_t HM = (int64_t)H * M;
  const T2* P = reinterpret_cast<const T2*>(ws + job.probe);
  const T2* V = reinterpret_cast<const T2*>(ws + job.wts);
  const int* rowflag = reinterpret_cast<const int*>(ws + job.rowflag);
  // probe rows p0 .. p0 + np - 1 = yb - uy_hi .. ye - 1 - uy_lo (inside [0, H))
  const int p0 = yb - job.uy_hi, np = nr + nuy - 1;
  for (int i = threadIdx.x; i < np; i += blockDim.x) ps[i] = P[(int64_t)(p0 + i) * rs];   // rs: probe row stride
  for (int i = threadIdx.x; i < (DM + 1) * nr; i += blockDim.x) {
    const int a = i / nr, r = i - a * nr;
    vs[a][r] = V[a * HM + (int64_t)(yb + r) * M];
  }
  for (int i = threadIdx.x; i < nr; i += blockDim.x) fl[i] = rowflag[yb + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T ysc = (T)2 / (T)(H > 1 ? H - 1 : 1);
  T dc[NMONO], nq[NMONO];
#pragma unroll
  for (int m = 0; m < NMONO; ++m) { dc[m] = 0; nq[m] = 0; }
  if (warp < nuy) {
    const int uy = job.uy_lo + warp;
    for (int r = lane; r < nr; r += 32) {
      if (!fl[r]) continue;
      const int y = yb + r;
      const T2 pv = ps[y - uy - p0];
      const T yt = (T)y * ysc - (T)1;
#pragma unroll
      for (int a = 0; a <= DM; ++a) {
        const T2 v = vs[a][r];
        const T d0 = v.x * pv.x, n0 = v.y * pv.y;
        T yp = 1;
#pragma unroll
        for (int b = 0; a + b <= DM; ++b) {
          dc[mono_index(a, b)] += yp * d0;
          nq[mono_index(a, b)] += yp * n0;
          yp *= yt;
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < NMONO; ++m) {
    const T s0 = warp_sum(dc[m]), s1 = warp_sum(nq[m]);
    if (lane == 0 && warp < nuy) { red[warp][m] = (double)s0; red[warp][NMONO + m] = (double)s1; }
  }
  __syncthreads();
  const double inv = 1.0 / (double)Nf;
  const int nux = job.ux_hi - job.ux_lo + 1;
  double* out = reinterpret_cast<double*>(ws + job.out);
  for (int i = threadIdx.x; i < nuy * nux * NMONO; i += blockDim.x) {
    const int m = i % NMONO, t = i / NMONO, iu = t / nux, ux = job.ux_lo + t % nux;
    const double v = red[iu][m] + ((ux & 1) ? -red[iu][NMONO + m] : red[iu][NMONO + m]);
    atomicAdd(out + ((job.uy_lo + iu + w) * L + (ux + w)) * NMONO + m, v * inv);
  }
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(sms, 1);
}

// Slot-0 sums of jobs job0 .. job0 + njobs - 1 (rs: row stride of the probe
// slabs), in bands of at most slot0_rows rows; a launch of few jobs takes
// shorter bands (at least 64 rows) for about four CTAs per SM.
template <typename T, int DM>
static cudaError_t slot0_T(const sfft_plan_s* p, int job0, int njobs, int rs, void* ws) {
  const int H = p->d.H, w = (p->d.L - 1) / 2, nrow = std::max(1, H - 2 * w);
  const int nb_want = (int)std::min<int64_t>((4 * (int64_t)sm_count() + njobs - 1) / njobs, 1 << 16);
  const int rows = std::min(slot0_rows<T>(), std::max(64, (nrow + nb_want - 1) / nb_want));
  const int nb = (nrow + rows - 1) / rows;
  k_contract_slot0<T, DM><<<dim3(njobs, nb), 32 * max_uy<T>(), 0, p->stream>>>(p->d_jobs + job0, (char*)ws, H, p->M,
                                                                                p->Nf, p->d.L, rs, rows);
  p->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T, int DM, int NS>
static cudaError_t contract_T(const sfft_plan_s* p, int job0, int njobs, int rows_per_cta, void* ws) {
  constexpr int KT = kt_for<T, DM>();
  const int H = p->d.H, L = p->d.L;
  constexpr int MU = max_uy<T>();
  const size_t smem = 2 * sizeof(Stage<T, DM, KT, MU>) + 32 + sizeof(T) * L * L * n_mono(DM);
  auto kern = k_contract<T, DM, KT, NS>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // A launch of few jobs (one CCD's KB or b_K block is a single job) shortens
  // its row bands until its CTAs fill the resident slots of the SMs: as many
  // bands as one wave holds, so that no CTA starts after the others finish.
  // Each band ends with a lag DFT over its k-slots, so a band keeps at least
  // 128 rows.
  const int nk = (p->M + KT - 1) / KT;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, cta_threads<T, DM, KT, NS>(), smem) != cudaSuccess) {
    (void)cudaGetLastError();   // a failed query leaves no error for the launches below to report
    occ = 1;
  }
  occ = std::max(occ, 1);
  const int64_t slots = (int64_t)occ * sm_count(), per_band = (int64_t)nk * njobs;
  if (per_band * ((H + rows_per_cta - 1) / rows_per_cta) < slots) {
    const int nb_fit = (int)std::max<int64_t>(1, slots / per_band);   // rounding rows up keeps the count <= this
    const int rows = ((H + nb_fit - 1) / nb_fit + kChunk - 1) / kChunk * kChunk;
    rows_per_cta = std::min(rows_per_cta, std::max(128, rows));
  }
  const int nb = (H + rows_per_cta - 1) / rows_per_cta;
  // row bands vary slowest: the CTAs in flight share one band of the weight
  // spectra (read by every job), which then stays in L2 across the jobs
  for (int j0 = 0; j0 < njobs; j0 += 65535) {   // grid.y limit
    dim3 grid((p->M + KT - 1) / KT, std::min(65535, njobs - j0), nb);
    kern<<<grid, cta_threads<T, DM, KT, NS>(), smem, p->stream>>>(p->d_jobs + job0 + j0, (char*)ws, H, p->M,
                                                                            p->Nf, L, rows_per_cta,
                                                                            (const c_t<T>*)p->twD, (const T*)p->ytab);
    p->nlaunch += 1;
  }
  return slot0_T<T, DM>(p, job0, njobs, p->M, ws);
}

cudaError_t launch_contract_slot0(const sfft_plan_s* p, int DM, int job0, int njobs, void* ws) {
  if (njobs <= 0) return cudaSuccess;
  const int rs = p->dl ? 16 : p->M;
  switch (DM) {
    case 0: return slot0_T<float, 0>(p, job0, njobs, rs, ws);
    case 2: return slot0_T<float, 2>(p, job0, njobs, rs, ws);
    case 4: return slot0_T<float, 4>(p, job0, njobs, rs, ws);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int NS>
static cudaError_t contract_dm(const sfft_plan_s* p, int DM, int job0, int njobs, int rows_per_cta, void* ws) {
  switch (DM) {
    case 0: return contract_T<T, 0, NS>(p, job0, njobs, rows_per_cta, ws);
    case 1: return contract_T<T, 1, NS>(p, job0, njobs, rows_per_cta, ws);
    case 2: return contract_T<T, 2, NS>(p, job0, njobs, rows_per_cta, ws);
    case 3: return contract_T<T, 3, NS>(p, job0, njobs, rows_per_cta, ws);
    case 4: return contract_T<T, 4, NS>(p, job0, njobs, rows_per_cta, ws);
    default: return cudaErrorInvalidValue;
  }
}

// lag_parts: threads sharing the lags of one (k-slot, monomial group), 2 or 3
// (FP32 only; the FP64 path always uses 2)
cudaError_t launch_contract(const sfft_plan_s* p, int DM, int job0, int njobs, int rows_per_cta, int lag_parts,
                            void* ws) {
  if (njobs <= 0) return cudaSuccess;
  if (p->fp64) return contract_dm<double, 2>(p, DM, job0, njobs, rows_per_cta, ws);
  if (lag_parts == 1) return contract_dm<float, 1>(p, DM, job0, njobs, rows_per_cta, ws);
  return lag_parts == 3 ? contract_dm<float, 3>(p, DM, job0, njobs, rows_per_cta, ws)
                        : contract_dm<float, 2>(p, DM, job0, njobs, rows_per_cta, ws);
}

}  // namespace sfft
