// Tensor-core lag contraction of the product spectra (FP32 path, KK block).
//
// For one k-slot the y sum of the lag contraction is a real matrix product:
//   C[(m, Re|Im)][(d, u_y)] = sum_{y, re|im} A[(m, Re|Im)][(y, re|im)] B[(y, re|im)][(d, u_y)]
// with W_m(y) = yt(y)^b V^_a(y, k) for monomial m = (a, b), the A rows
// (Re: W_r, W_i) and (Im: -W_i, W_r), and B = (P_r, P_i)(y - u_y, k) for the
// offset difference d, so that C = sum_y conj(W_m) P^_d(y - u_y): exactly the
// C_{a,b}(u_y, k) of the FP32 FMA kernel.  The lag DFT over k and the FP64
// accumulation into G follow as there.
//
// Each operand x is split as x = hi + lo with hi the TF32 truncation of x and
// lo = x - hi (exact in FP32); the product x y is taken as hi_x hi_y on the
// TF32 tensor cores (m16n8k8: exact product, FP32 accumulation) plus the
// correction bf16(hi_x) bf16(lo_y) + bf16(lo_x) bf16(y) on the BF16 tensor
// cores (m16n8k16: both corrections of four rows in one instruction).  This is
// the split-operand scheme of Ootomo and Yokota (2022), which recovers
// single-precision products from low-precision tensor-core inputs, with the
// two small terms carried in BF16 (each is about 2^-10 of the product and
// keeps 8 bits), for a product error within about 2^-18.
//
// Work decomposition: a CTA owns KT consecutive k-slots (one warp each), one
// band of weight rows and one "pattern": up to NP = 8 NT consecutive (d, u_y)
// pairs of the d-batch's pair list, which is ordered by d then u_y.  A warp
// keeps C for its k-slot, every monomial (16-row tiles) and the pattern's NT
// 8-column tiles in registers.  Rows arrive in chunks of kChunkTC through
// bulk copies into two alternating shared-memory stages: for every difference
// of the pattern the probe rows z = y - u_y of the chunk (kChunkTC + n_lag - 1
// rows of KT slots), the weight rows of every exponent a and the powers of yt.
// Slot 0 (the packed real bins) is dropped at the flush and summed exactly by
// k_contract_slot0, as in the FMA kernel.
#include "bulk.cuh"
#include "common.cuh"
#include "plan.h"

namespace sfft {

namespace {

constexpr int kChunkTC = kTcChunk;   // 4 mma k-steps of 4 rows

template <int DM> __host__ __device__ constexpr int n_mtiles() { return (n_mono(DM) + 7) / 8; }

// Probe rows per stage: sum over the pattern's differences of (kChunkTC + n_lag - 1).
template <int KT, int CAP> struct TcStage {
  static constexpr int RS = KT + 2;   // float2 per staged row: KT slots + 16 bytes of padding (bank spread)
  float2 P[CAP][RS];
  float2 V[kMaxWeightDeg + 1][kChunkTC][RS];
  float ypw[kChunkTC][16];            // yt^b as duplicated pairs (the FP32 power table's 64-byte rows)
};

// hi: the sign, exponent and ten leading mantissa bits of x (a TF32 value)
__device__ __forceinline__ float tf32_trunc(float x) { return __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

// two floats rounded to BF16 and packed, `lo` in the low half (the lower matrix index)
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mono_ab(int m, int& a, int& b) {
  int n = 0;
  while ((n + 1) * (n + 2) / 2 <= m) ++n;
  b = m - n * (n + 1) / 2;
  a = n - b;
}

// Issue the bulk copies of rows [yc, ye) into stage `st`, counted on `full`:
// warp w copies the probe rows of the pattern's differences w, w + nwarp, ...
// (lane i row i), then all threads copy the weight rows and thread 0 the powers of yt.
template <int DM, int KT, int CAP>
__device__ __forceinline__ void tc_produce(TcStage<KT, CAP>& st, uint64_t* full, const char* __restrict__ probe,
                                           int64_t slab, const float2* __restrict__ V, const float* __restrict__ ytab,
                                           const int4* __restrict__ dj, int nd, int npair, int64_t HM, int M, int k0,
                                           int yc, int ye) {
  constexpr unsigned seg = KT * sizeof(float2);
  const int nrow = ye - yc;
  const int nprobe = nd * (nrow - 1) + npair;   // sum over differences of nrow + n_lag - 1
  const int nv = (DM + 1) * nrow;
  if (threadIdx.x == 0) mbar_arrive_expect_tx(full, seg * (unsigned)(nprobe + nv) + (unsigned)(nrow * 64));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int i = warp; i < nd; i += nwarp) {
    const int4 e = dj[i];   // (d_local, u_lo, u_hi, row_base)
    const int rows = nrow + e.z - e.y;
    const char* src = probe + (int64_t)e.x * slab;
    for (int r = lane; r < rows; r += 32) {
      const int z = yc - e.z + r;
      bulk_copy_g2s(&st.P[e.w + r][0], src + ((int64_t)z * M + k0) * (int64_t)sizeof(float2), seg, full);
    }
  }
  for (int t = threadIdx.x; t < nv; t += blockDim.x) {
    const int a = t / nrow, yy = t - a * nrow;
    bulk_copy_g2s(&st.V[a][yy][0], V + a * HM + (int64_t)(yc + yy) * M + k0, seg, full);
  }
  if (threadIdx.x == 0) bulk_copy_g2s(&st.ypw[0][0], ytab + (int64_t)yc * 16, (unsigned)(nrow * 64), full);
}

}  // namespace

template <int DM, int KT, int NT, int CAP>
__global__ void __launch_bounds__(KT * 32, 2)
k_contract_tc(const TcJob* __restrict__ jobs, const int4* __restrict__ pairs, const int4* __restrict__ djobs,
              char* __restrict__ ws, int H, int M, int Nf, int L, int rows_per_cta, int64_t slab,
              const float2* __restrict__ twD, const float* __restrict__ ytab) {
  constexpr int NMT = n_mtiles<DM>();
  constexpr int NMONO = n_mono(DM);
  constexpr int NP = 8 * NT;
  using St = TcStage<KT, CAP>;
  constexpr int RS = St::RS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  St* stages = reinterpret_cast<St*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + 2 * sizeof(St));        // [2]
  float2* tw = reinterpret_cast<float2*>(smem_raw + 2 * sizeof(St) + 16);         // [KT][kMaxL]
  float* red = reinterpret_cast<float*>(smem_raw);                                // aliases the stages at the flush

  const TcJob job = jobs[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int w = (L - 1) / 2;
  const int k0 = blockIdx.x * KT, kk = warp, k = k0 + kk;
  const int4* dj = djobs + job.dj0;
  const int4* pr = pairs + job.pair0;

  // stages start zeroed so that rows past a ragged chunk end read finite values
  for (int i = threadIdx.x; i < (int)(2 * sizeof(St) / 16); i += blockDim.x)
    reinterpret_cast<float4*>(smem_raw)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  int y0 = blockIdx.z * rows_per_cta, y1 = y0 + rows_per_cta;
  if (y0 < w) y0 = w;
  if (y1 > H - w) y1 = H - w;
  const int64_t HM = (int64_t)H * M;
  const char* probe = ws + job.probe;
  const float2* V = reinterpret_cast<const float2*>(ws + job.wts);

  // per-thread operand coordinates: monomials (A rows g, g + 8 of each 16-row tile)
  int am[NMT], bm[NMT];
  bool vm[NMT];
#pragma unroll
  for (int m = 0; m < NMT; ++m) {
    const int ab = m * 8 + g;
    vm[m] = ab < NMONO;
    mono_ab(vm[m] ? ab : 0, am[m], bm[m]);
  }
  // B column g of each 8-column tile: the staged probe row of (d, u_y) for row t of a k-step
  int poff[NT];
#pragma unroll
  for (int n = 0; n < NT; ++n) {
    int q = n * 8 + g;
    if (q >= job.npair) q = 0;   // padding columns read pair 0; their results are dropped
    const int4 pq = pr[q];       // (d_local, u_y, ux_lo, ux_hi)
    int row = 0;
    for (int i = 0; i < job.nd; ++i)
      if (dj[i].x == pq.x) row = dj[i].w + t - pq.y + dj[i].z;
    poff[n] = row * RS + kk;
  }
  // 8-column tiles that hold at least one pair (warp-uniform)
  const int nt_live = (job.npair + 7) / 8;

  float acc[NMT][NT][4];
#pragma unroll
  for (int m = 0; m < NMT; ++m)
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[m][n][c] = 0.f;

  const int nchunk = y1 > y0 ? (y1 - y0 + kChunkTC - 1) / kChunkTC : 0;
  if (nchunk > 0)
    tc_produce<DM, KT, CAP>(stages[0], &full[0], probe, slab, V, ytab, dj, job.nd, job.npair, HM, M, k0, y0,
                       min(y0 + kChunkTC, y1));
  for (int c = 0; c < nchunk; ++c) {
    const int yc = y0 + c * kChunkTC, ye = min(yc + kChunkTC, y1);
    if (c + 1 < nchunk) {   // stage (c+1)&1 was released by the barrier that closed chunk c - 1
      const int yn = yc + kChunkTC;
      tc_produce<DM, KT, CAP>(stages[(c + 1) & 1], &full[(c + 1) & 1], probe, slab, V, ytab, dj, job.nd, job.npair, HM,
                         M, k0, yn, min(yn + kChunkTC, y1));
    }
    const bool landed = mbar_wait_bounded(&full[c & 1], (unsigned)((c >> 1) & 1));
    if (!__syncthreads_and(landed)) {
      if (threadIdx.x == 0) atomicOr(reinterpret_cast<int*>(ws + job.status), 4);
      if (c + 1 < nchunk) mbar_wait_bounded(&full[(c + 1) & 1], (unsigned)(((c + 1) >> 1) & 1));
      return;
    }
    const St& st = stages[c & 1];
    const float2* P0 = &st.P[0][0];
#pragma unroll 2
    for (int s = 0; s < kChunkTC / 4; ++s) {
      const int r = 4 * s + t;
      const bool rv = yc + r < ye;
      // A fragments.  TF32, k = (row t: re, im) at columns (t, t + 4):
      //   (a0, a1, a2, a3) = rows (g, g + 8) x columns (t, t + 4) = (W_r, -W_i, W_i, W_r) of hi(W).
      // BF16, k = 2t + c (c = re, im) for the first correction and 8 + 2t + c for the second:
      //   rows g (Re) and g + 8 (Im) hold (lo_r, lo_i), (-lo_i, lo_r), (W_r, W_i), (-W_i, W_r).
      uint32_t wt[NMT][3], wb[NMT][4];
#pragma unroll
      for (int m = 0; m < NMT; ++m) {
        const float2 v = st.V[am[m]][r][kk];
        const float yp = st.ypw[r][2 * bm[m]];
        const bool on = rv && vm[m];
        const float wr = on ? yp * v.x : 0.f, wi = on ? yp * v.y : 0.f;
        const float hr = tf32_trunc(wr), hi = tf32_trunc(wi);
        const float lr = wr - hr, li = wi - hi;
        wt[m][0] = __float_as_uint(hr);
        wt[m][1] = __float_as_uint(hi);
        wt[m][2] = __float_as_uint(-hi);
        wb[m][0] = pack_bf16(lr, li);
        wb[m][1] = pack_bf16(-li, lr);
        wb[m][2] = pack_bf16(wr, wi);
        wb[m][3] = pack_bf16(-wi, wr);
      }
      // two column tiles at a time: the two products of four independent
      // accumulators interleave, so no MMA waits on the previous one
#pragma unroll
      for (int n = 0; n < NT; n += 2) {
        if (n >= nt_live) break;
        uint32_t bt[2][2], bb[2][2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float2 pv = P0[poff[n + e] + 4 * s * RS];
          const float hr = tf32_trunc(pv.x), hi = tf32_trunc(pv.y);
          bt[e][0] = __float_as_uint(hr);
          bt[e][1] = __float_as_uint(hi);
          bb[e][0] = pack_bf16(hr, hi);                  // k = 2t, 2t + 1: hi(P) (multiplies lo(W))
          bb[e][1] = pack_bf16(pv.x - hr, pv.y - hi);    // k = 8 + 2t, 9 + 2t: lo(P) (multiplies W)
        }
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
          for (int m = 0; m < NMT; ++m)
            mma_bf16(acc[m][n + e], wb[m][0], wb[m][1], wb[m][2], wb[m][3], bb[e][0], bb[e][1]);
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
          for (int m = 0; m < NMT; ++m)
            mma_tf32(acc[m][n + e], wt[m][0], wt[m][2], wt[m][1], wt[m][0], bt[e][0], bt[e][1]);
      }
    }
    __syncthreads();
  }

  // ---- flush: lag DFT over the CTA's k-slots into shared FP32 sums (fixed
  // order), then FP64 atomics
  constexpr int RM = 8 * NMT + 1;   // monomials per (pair, u_x) entry, padded against bank conflicts
  const int nred = NP * L * RM;
  for (int i = threadIdx.x; i < nred; i += blockDim.x) red[i] = 0.f;
  if (lane < L) {
    const int ux = lane - w;
    int idx = (int)(((int64_t)k * ux) % Nf);
    if (idx < 0) idx += Nf;
    const float2 cs = twD[idx];
    tw[kk * kMaxL + lane] = make_float2(2.f * cs.x, 2.f * cs.y);
  }
  __syncthreads();
  // the warps add their k-slot's terms in turn (a fixed order, so the sums do
  // not depend on scheduling); within a warp every lane owns distinct entries
  for (int turn = 0; turn < KT; ++turn) {
    if (warp == turn && k != 0 && k < M) {   // slot 0: the packed real bins, summed by k_contract_slot0
#pragma unroll
      for (int n = 0; n < NT; ++n) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int q = n * 8 + 2 * t + j;
          if (q >= job.npair) continue;
          const int4 pq = pr[q];
#pragma unroll
          for (int m = 0; m < NMT; ++m) {
            if (!vm[m]) continue;
            const float cr = acc[m][n][j], ci = acc[m][n][2 + j];
            float* dst = red + (q * L + w) * RM + m * 8 + g;
            for (int ux = pq.z; ux <= pq.w; ++ux) {
              const float2 c2 = tw[kk * kMaxL + ux + w];
              atomicAdd(dst + ux * RM, cr * c2.x + ci * c2.y);   // one add per entry per turn
            }
          }
        }
      }
    }
    __syncthreads();
  }
  const double inv = 1.0 / (double)Nf;
  double* out = reinterpret_cast<double*>(ws + job.out);
  const int LL = L * L;
  for (int q = warp; q < job.npair; q += KT) {   // one pair per warp: its (u_x, monomial) entries over the lanes
    const int4 pq = pr[q];
    const int nval = (pq.w - pq.z + 1) * NMONO;
    double* o = out + ((int64_t)pq.x * LL + (pq.y + w) * L + (pq.z + w)) * NMONO;
    const float* rq = red + (q * L + pq.z + w) * RM;
    for (int e = lane; e < nval; e += 32) {
      const int iu = e / NMONO, mono = e - iu * NMONO;
      const float v = rq[iu * RM + mono];
      if (v != 0.f) atomicAdd(o + e, (double)v * inv);
    }
  }
}

template <int DM, int NT, int CAP>
static cudaError_t contract_tc_dm(const sfft_plan_s* p, int job0, int njobs, void* ws) {
  constexpr int KT = kTcKT;
  const size_t smem = 2 * sizeof(TcStage<KT, CAP>) + 16 + sizeof(float2) * KT * kMaxL;
  static_assert(sizeof(float) * (n_mtiles<DM>() * 8 + 1) * 8 * NT * kMaxL <= 2 * sizeof(TcStage<KT, CAP>),
                "flush sums must fit in the stage memory");
  auto kern = k_contract_tc<DM, KT, NT, CAP>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);   // two CTAs per SM
  const int H = p->d.H;
  const int rows = p->tc_rows;
  const int nb = (H + rows - 1) / rows;
  const int64_t slab = (int64_t)H * p->M * (int64_t)sizeof(float2);
  for (int j0 = 0; j0 < njobs; j0 += 65535) {
    dim3 grid(p->M / KT, std::min(65535, njobs - j0), nb);
    kern<<<grid, KT * 32, smem, p->stream>>>(p->d_tcjobs + job0 + j0, p->d_tcpairs, p->d_tcdj, (char*)ws, H, p->M,
                                             p->Nf, p->d.L, rows, slab, (const float2*)p->twD,
                                             (const float*)p->ytab);
    p->nlaunch += 1;
  }
  return cudaGetLastError();
}

cudaError_t launch_contract_tc(const sfft_plan_s* p, int batch_index, int c0, int nc, void* ws) {
  // jobs are ordered CCD-major with the same count per CCD: the group's jobs are one run
  const int per_ccd = p->tc_count[batch_index] / p->d.batch;
  const int job0 = p->tc_first[batch_index] + c0 * per_ccd, njobs = nc * per_ccd;
  if (njobs <= 0) return cudaSuccess;
  switch (p->DM_KK) {
    case 0: return contract_tc_dm<0, kTcNT, kTcRowCap>(p, job0, njobs, ws);
    case 2: return contract_tc_dm<2, kTcNT, kTcRowCap>(p, job0, njobs, ws);
    case 4: return contract_tc_dm<4, kTcNT, kTcRowCap>(p, job0, njobs, ws);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sfft
