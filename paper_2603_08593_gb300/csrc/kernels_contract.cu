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

template <typename T, int DM, int KT, int G>
__device__ __forceinline__ void contract_group(const CJob& job, const char* __restrict__ ws, int k, int y0, int y1,
                                               int H, int M, int Nf, int L, T* red,
                                               const c_t<T>* __restrict__ twD) {
  using T2 = c_t<T>;
  using C = GroupCfg<DM, G>;
  constexpr int NS = C::NLO + C::NHI;
  constexpr int MU = max_uy<T>();
  const int lane = threadIdx.x & 31;
  const int nuy = job.uy_hi - job.uy_lo + 1;
  T2 acc[MU][NS];
#pragma unroll
  for (int i = 0; i < MU; ++i)
#pragma unroll
    for (int s = 0; s < NS; ++s) { acc[i][s].x = 0; acc[i][s].y = 0; }

  const int64_t HM = (int64_t)H * M;
  const T2* __restrict__ P = reinterpret_cast<const T2*>(ws + job.probe) + k;
  const T2* __restrict__ Vlo = reinterpret_cast<const T2*>(ws + job.wts) + C::ALO * HM + k;
  const T2* __restrict__ Vhi = reinterpret_cast<const T2*>(ws + job.wts) + C::AHI * HM + k;
  const int* __restrict__ rowflag = reinterpret_cast<const int*>(ws + job.rowflag);
  const bool slot0 = (k == 0);
  const T ysc = (T)2 / (T)(H > 1 ? H - 1 : 1);

  for (int y = y0; y < y1; ++y) {
    if (!rowflag[y]) continue;
    const T2 vl = Vlo[(int64_t)y * M];
    const T l1 = vl.x, l2 = slot0 ? (T)0 : vl.y, l3 = slot0 ? vl.y : vl.x, l4 = slot0 ? (T)0 : -vl.y;
    T h1 = 0, h2 = 0, h3 = 0, h4 = 0;
    if constexpr (C::NHI > 0) {
      const T2 vh = Vhi[(int64_t)y * M];
      h1 = vh.x; h2 = slot0 ? (T)0 : vh.y; h3 = slot0 ? vh.y : vh.x; h4 = slot0 ? (T)0 : -vh.y;
    }
    const T yt = (T)y * ysc - (T)1;
    T yp[5];
    yp[0] = 1;
#pragma unroll
    for (int b = 1; b < 5; ++b) yp[b] = yp[b - 1] * yt;
    const T2* prow = P + (int64_t)(y - job.uy_lo) * M;
#pragma unroll
    for (int iu = 0; iu < MU; ++iu) {
      if (iu < nuy) {
        const T2 pv = prow[-(int64_t)iu * M];
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

  // lag DFT over this thread's k, then reduce over the warp's 32 k-slots
  const int w = (L - 1) / 2;
  constexpr int NMONO = n_mono(DM);
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
  extern __shared__ __align__(8) unsigned char red_raw[];
  T* red = reinterpret_cast<T*>(red_raw);   // [L][L][n_mono(DM)]
  constexpr int NMONO = n_mono(DM);
  const CJob job = jobs[blockIdx.z];
  const int nred = L * L * NMONO;
  for (int i = threadIdx.x; i < nred; i += blockDim.x) red[i] = (T)0;
  __syncthreads();
  const int w = (L - 1) / 2;
  const int g = threadIdx.x / KT;
  const int k = blockIdx.x * KT + (threadIdx.x % KT);
  int y0 = blockIdx.y * rows_per_cta, y1 = y0 + rows_per_cta;
  if (y0 < w) y0 = w;
  if (y1 > H - w) y1 = H - w;
  if (k < M) {
    if (g == 0) contract_group<T, DM, KT, 0>(job, ws, k, y0, y1, H, M, Nf, L, red, twD);
    if constexpr (n_groups<DM>() > 1) { if (g == 1) contract_group<T, DM, KT, 1>(job, ws, k, y0, y1, H, M, Nf, L, red, twD); }
    if constexpr (n_groups<DM>() > 2) { if (g == 2) contract_group<T, DM, KT, 2>(job, ws, k, y0, y1, H, M, Nf, L, red, twD); }
  }
  __syncthreads();
  const double inv = 1.0 / (double)Nf;
  const int nuy = job.uy_hi - job.uy_lo + 1, nux = job.ux_hi - job.ux_lo + 1;
  const int nval = nuy * nux * NMONO;
  for (int i = threadIdx.x; i < nval; i += blockDim.x) {
    const int m = i % NMONO, t = i / NMONO;
    const int ux = job.ux_lo + t % nux, uy = job.uy_lo + t / nux;
    const int ridx = ((uy + w) * L + (ux + w)) * NMONO + m;
    const T v = red[ridx];
    if (v != (T)0) atomicAdd(reinterpret_cast<double*>(ws + job.out) + ridx, (double)v * inv);
  }
}

template <typename T, int DM>
static cudaError_t contract_T(const sfft_plan_s* p, int job0, int njobs, int rows_per_cta, int ktile, void* ws) {
  const int H = p->d.H, L = p->d.L;
  const size_t smem = sizeof(T) * L * L * n_mono(DM);
  const int nb = (H + rows_per_cta - 1) / rows_per_cta;
  if (ktile == 64) {
    constexpr int KT = 64;
    dim3 grid((p->M + KT - 1) / KT, nb, njobs);
    k_contract<T, DM, KT><<<grid, KT * n_groups<DM>(), smem, p->stream>>>(p->d_jobs + job0, (char*)ws, H, p->M, p->Nf, L, rows_per_cta,
                                                                          (const c_t<T>*)p->twD);
  } else {
    constexpr int KT = 128;
    dim3 grid((p->M + KT - 1) / KT, nb, njobs);
    k_contract<T, DM, KT><<<grid, KT * n_groups<DM>(), smem, p->stream>>>(p->d_jobs + job0, (char*)ws, H, p->M, p->Nf, L, rows_per_cta,
                                                                          (const c_t<T>*)p->twD);
  }
  p->nlaunch += 1;
  return cudaGetLastError();
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
