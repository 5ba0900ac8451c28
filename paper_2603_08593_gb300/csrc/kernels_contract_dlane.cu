// Lag contraction of the product spectra on the tcgen05 tensor cores with one
// tensor-memory lane per offset difference (FP32 path, KK block).
//
// For one k-slot the y sum
//   C[d][u_y][(m, Re|Im)] = sum_y conj(W_m(y)) P^_d(y - u_y)
//                         = sum_{y'} P^_d(y') conj(W_m(y' + u_y))
// is, for each u_y, a real matrix product whose rows are the differences d
// of a tile (128 lanes), whose columns are the monomials (Re 0..15, Im
// 16..31) and whose inner dimension runs over the rows y' and (re, im).  The
// A operand (the probe rows) is the same for every u_y; only the weight rows
// shift.  So each probe value is split and stored to tensor memory once, and
// one MMA of N = 32 nu columns covers all nu u_y of a CTA: its B operand is
// read from weight-row blocks laid out so that the n-groups of consecutive
// u_y are consecutive 128-byte core matrices.  Block q (1024 bytes) holds the
// row pair (2q, 2q + 1) for the 32 columns n (four 128-byte core matrices,
// "even") and then the pair (2q + 1, 2q + 2) (four more, "odd"); with the
// n-group stride at 128 bytes and the K stride (one row pair) at 1024 bytes,
// the n-groups of u_y index i start at row 4 j + i of the k-step j (even
// part of block 2 j + i / 2 for even i, odd part for odd i).  The products are
// split as in kernels_contract_umma.cu (hi_x hi_y on kind::tf32, K = 8 = four
// rows, plus bf16(hi_x) bf16(lo_y) + bf16(lo_x) bf16(y) on kind::f16, K = 16;
// Ootomo and Yokota, 2022), with the BF16 inner order (row pair, row parity,
// hi/lo part, re/im) so that a row pair is one 16-byte column there too.
//
// A CTA takes two adjacent k-slots and up to NU consecutive u_y of one tile
// over all weight rows of the band; its 2 x NU accumulators (32 FP32 columns
// each) stay in tensor memory and go to an HBM buffer C[k][d][u_y][32] at the
// end.  k_lag_dft (kernels_lag_dft.cu) then forms the lags u_x of every
// (d, u_y) pair, with FP32 sums within a warp and FP64 across its warps.
//
// Roles (704 threads, one CTA per SM):
//   warps 0-15 A producers: lane l of warp w is difference 32 (w % 4) + l of
//              the tile (tensor-memory lane 32 (w % 4) + l); warp group w / 4
//              takes k-step w / 4 (four rows y') of every chunk, so that four
//              k-steps' stores to tensor memory are in flight at once; one
//              16-byte load per row gives both k-slots' probe values, split
//              into 2 x 16 A columns (tcgen05.st); warps 0-3 then run the
//              epilogue;
//   warps 16-19 B producers: the weight-row blocks (TF32 and BF16) of both
//              k-slots for each staged chunk of 16 rows y', every row written
//              to its even and its odd block, a half-warp filling one 128-byte
//              core matrix per store;
//   warp 20    MMA issuer: per pair of k-steps and k-slot, four MMAs of
//              N = 32 nu (TF32 and BF16 of both k-steps) back to back;
//   warp 21    copy producer: per chunk one tensor-map box of probe rows
//              (128 differences x 17 rows x 2 slots, from the k-slot-blocked
//              product spectra [d][k / 16][y][k % 16]), one box of weight rows
//              per exponent and the powers of yt.
// Every wait is bounded; a wait that gives up flags the CCD (status bit 4)
// and makes every role leave its loop, after which the issued copies and
// MMAs are drained (bounded) and the tensor memory is freed.
#include <cuda.h>

#include "bulk.cuh"
#include "common.cuh"
#include "plan.h"
#include "umma_common.cuh"

namespace sfft {

namespace {

constexpr int CH = kDlChunk;          // rows y' per staged chunk
constexpr int KSC = CH / 4;           // k-steps per chunk
constexpr int NU = kDlMaxU;           // u_y per CTA at most
constexpr int GA = 4;                 // k-steps of A operands in flight
constexpr int NST = 3;                // staged chunks of probe and weight rows in flight
constexpr int PBR = CH + 1;           // probe rows per box: a spare row staggers the lanes' banks
constexpr int PBYTES = 128 * PBR * 16;
constexpr int VR = CH + NU;           // weight rows per box (CH + NU - 1 used)
constexpr int VSLOT = (VR * 16 + 127) / 128 * 128;
constexpr int NQ = (4 * (KSC - 1) + NU - 1) / 2 + 2;   // weight-row blocks (row pairs) per chunk
constexpr int QB = 1024;              // bytes per block: even and odd row pairs of the 32 columns n
constexpr int WBLK = NQ * QB;         // bytes of one chunk's blocks per k-slot and operand format
constexpr int WARP_BP = 16;           // first B-producer warp (warps 0-15: A producers, one k-step of a chunk each)
constexpr int WARP_MMA = 20, WARP_COPY = 21;
constexpr int NTHREADS = 32 * 22;
static_assert(WARP_BP / 4 == KSC, "one A-producer warp group per k-step of a chunk");
constexpr int TMEM_COLS = 512;        // D: 2 x NU x 32 columns, A: GA x 32 columns
static_assert(2 * NU * 32 + GA * 32 <= TMEM_COLS, "tensor memory budget");
static_assert(CH % 8 == 0 && VR % 2 == 0 && GA % 2 == 0, "chunk geometry: k-steps in pairs");

struct DStage {
  uint8_t P[PBYTES];                       // [difference][row y'][2 slots]
  uint8_t V[kMaxWeightDeg + 1][VSLOT];     // per exponent a: [row][2 slots]
  float ypw[VR][16];                       // yt^b of the weight rows (pairs (yt^b, yt^b), b = 0..4)
};
static_assert(PBYTES % 128 == 0 && sizeof(DStage) % 128 == 0, "tensor copy alignment");

struct DSmem {
  DStage st[NST];
  uint8_t wblk[2][2][2][WBLK];     // [stage][slot][TF32, BF16] weight-row blocks
  uint64_t raw_full[NST], raw_empty[NST], strip_full[2], strip_empty[2];
  uint64_t a_full[GA], a_empty[GA], done;
  uint32_t tmem_base;
  int abort;
};

// Wait attribution (compile with -DSFFT_DLANE_WAIT_PROFILE): lane 0 of every
// warp adds the cycles it spends in each kind of wait, and the CTA's total
// cycles, to a device array that sfft_debug_contract_waits reads.  The
// default build compiles none of it.
enum WaitKind {
  W_COPY_RAW_EMPTY = 0,   // copy warp: a stage of probe rows to be released
  W_A_RAW_FULL,           // A producers: probe rows to land
  W_A_SLOT_EMPTY,         // A producers: an A slot in tensor memory to be consumed
  W_A_STORE,              // A producers: their tensor-memory stores to complete
  W_B_RAW_FULL,           // B producers: weight rows to land
  W_B_BLK_EMPTY,          // B producers: a stage of weight-row blocks to be consumed
  W_MMA_BLK_FULL,         // MMA issuer: weight-row blocks
  W_MMA_A_FULL,           // MMA issuer: A operands
  W_CTA_CYCLES,           // per CTA: cycles from setup to the epilogue
  W_NKIND
};
#ifdef SFFT_DLANE_WAIT_PROFILE
__device__ unsigned long long g_dl_wait[W_NKIND];
#define DL_T0() long long dl_t0_ = clock64()
#define DL_ACC(acc, kind) (acc)[kind] += clock64() - dl_t0_
#else
#define DL_T0() \
  do {          \
  } while (0)
#define DL_ACC(acc, kind) \
  do {                    \
  } while (0)
#endif

}  // namespace

template <int DM>
__global__ void __launch_bounds__(NTHREADS, 1)
k_contract_dlane(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmPs,
                 const __grid_constant__ CUtensorMap tmV, const DlJob* __restrict__ jobs, char* __restrict__ ws,
                 int H, int L, int dstride, int pz, int pzs, const float* __restrict__ ytab) {
  constexpr int NMONO = n_mono(DM);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  DSmem& S = *reinterpret_cast<DSmem*>(smem_raw);
  volatile int* abort = &S.abort;

  // grid (job within the CCD, slot pair, CCD): the CTAs of one k-slot block
  // (four slot pairs) and of both u_y runs of a tile run side by side and
  // share the block rows in L2
  const DlJob job = jobs[blockIdx.z * gridDim.x + blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = (L - 1) / 2;
  const int k0 = 2 * blockIdx.y;
  // weight rows of the band (M_fit vanishes within w of the edges)
  const int y0 = job.y_lo, y1 = job.y_hi;
  (void)w;
  const int ulo = job.u_lo, nu = job.nu;
  const int Ys = y0 - (ulo + nu - 1);           // first row y' any u_y of the CTA needs
  const int nchunk = y1 > y0 ? (y1 - ulo - Ys + CH - 1) / CH : 0;
  const int nstep = nchunk * KSC;
  // ---- setup: zeroed stages (lanes past the tile read zeros), barriers, tensor memory
  for (int i = threadIdx.x; i < (int)(sizeof(DStage) * NST / 16); i += NTHREADS)
    reinterpret_cast<float4*>(&S.st[0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&S.raw_full[i], 1);
      mbar_init(&S.raw_empty[i], WARP_BP + 4);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.strip_full[i], 4);
      mbar_init(&S.strip_empty[i], 1);
    }
    for (int i = 0; i < GA; ++i) { mbar_init(&S.a_full[i], 4); mbar_init(&S.a_empty[i], 1); }
    mbar_init(&S.done, 1);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "n"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = S.tmem_base;
  const uint32_t t_d = tbase;                  // accumulators: (slot s, u index i) at columns 32 (NU s + i)
  const uint32_t t_a = tbase + 2 * NU * 32;    // A: k-step slot g at columns 32 g + 16 s (TF32 0-7, BF16 8-15)

  int issued_chunks = 0;   // copy warp: chunks whose copies were issued
#ifdef SFFT_DLANE_WAIT_PROFILE
  long long wt[W_NKIND] = {};
  const long long cta_t0 = clock64();
#endif
  // a tile of at most pzs differences takes the smaller probe box (its other
  // lanes keep the zeros of the setup)
  const bool small_box = job.nlanes <= pzs;
  const int pzj = small_box ? pzs : pz;

  if (warp == WARP_COPY) {
    for (int c = 0; c < nchunk; ++c) {
      const int sidx = c % NST;
      {
        DL_T0();
        const bool ok_w = c < NST || wait_phase(&S.raw_empty[sidx], (unsigned)(((c / NST) - 1) & 1), abort);
        DL_ACC(wt, W_COPY_RAW_EMPTY);
        if (!ok_w) break;
      }
      DStage& st = S.st[sidx];
      const int yc = Ys + c * CH;
      // powers of yt for the weight rows inside the image (the others are masked)
      const int ylo = max(yc + ulo, 0), yhi = min(yc + ulo + VR, H);
      const unsigned ybytes = yhi > ylo ? (unsigned)(yhi - ylo) * 64u : 0u;
      if (lane == 0)
        mbar_arrive_expect_tx(&S.raw_full[sidx], (unsigned)(pzj * PBR * 16 + (DM + 1) * VR * 16) + ybytes);
      __syncwarp();
      if (lane == 0) {
        tma_load_4d(&st.P[0], small_box ? &tmPs : &tmP, 2 * (k0 & 15), yc, k0 >> 4, job.zp + job.d_first,
                    &S.raw_full[sidx]);
      } else if (lane <= DM + 1) {
        const int a = lane - 1;
        tma_load_3d(&st.V[a][0], &tmV, 2 * k0, yc + ulo, job.zw + a, &S.raw_full[sidx]);
      } else if (lane == 31 && ybytes > 0) {
        bulk_copy_g2s(&st.ypw[ylo - (yc + ulo)][0], ytab + (int64_t)ylo * 16, ybytes, &S.raw_full[sidx]);
      }
      issued_chunks = c + 1;
      __syncwarp();
    }
  } else if (warp == WARP_MMA) {
    // one MMA per k-step, k-slot and operand format covers the nu u_y of the
    // CTA: N = 32 nu columns, n-groups 128 bytes apart, row pairs 1024 apart
    const uint32_t id_tf32 = instr_desc(2, 32 * nu), id_bf16 = instr_desc(1, 32 * nu);
    const uint64_t dblk0 = smem_desc_kn(smem_u32(&S.wblk[0][0][0][0]), QB, 128);
    for (int c = 0; c < nchunk && !*abort; ++c) {
      const int sidx = c & 1;
      {
        DL_T0();
        const bool ok_w = wait_phase(&S.strip_full[sidx], (unsigned)((c >> 1) & 1), abort);
        DL_ACC(wt, W_MMA_BLK_FULL);
        if (!ok_w) break;
      }
      uint64_t dw[2][2];   // descriptors of the stage's blocks: [slot][TF32, BF16]
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int f = 0; f < 2; ++f) dw[s][f] = dblk0 + (uint64_t)((((sidx * 2 + s) * 2 + f) * WBLK) >> 4);
      bool live = true;
      // k-steps in pairs: each k-slot's accumulators take TF32 (j), BF16 (j),
      // TF32 (j + 1), BF16 (j + 1) back to back
      for (int j = 0; j < KSC; j += 2) {
        const int g = c * KSC + j, as = g % GA;   // k-steps g, g + 1 in A slots as, as + 1
        DL_T0();
        const bool ok_a = wait_phase(&S.a_full[as], (unsigned)((g / GA) & 1), abort) &&
                          wait_phase(&S.a_full[as + 1], (unsigned)(((g + 1) / GA) & 1), abort);
        DL_ACC(wt, W_MMA_A_FULL);
        if (!ok_a) {
          live = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (elect_one()) {
          const uint32_t acc = g > 0 ? 1u : 0u;   // the first k-step starts the accumulators
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const uint32_t dcol = t_d + 32 * NU * s;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint32_t acol = t_a + 32 * (as + h) + 16 * s;
              const uint64_t koff = (uint64_t)((2 * (j + h) * QB) >> 4);   // block 2 (j + h): rows 4 (j + h) ..
              asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                           " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                           ::"r"(dcol), "r"(acol), "l"(dw[s][0] + koff), "r"(id_tf32), "r"(h ? 1u : acc) : "memory");
              asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                           " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
                           ::"r"(dcol), "r"(acol + 8), "l"(dw[s][1] + koff), "r"(id_bf16), "r"(1u) : "memory");
            }
          }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       ::"r"(smem_u32(&S.a_empty[as])) : "memory");
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                       ::"r"(smem_u32(&S.a_empty[as + 1])) : "memory");
        }
        __syncwarp();
      }
      if (!live) break;
      if (elect_one())
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&S.strip_empty[sidx])) : "memory");
      __syncwarp();
    }
    // every MMA issued so far completes before the accumulators are read or freed
    if (elect_one())
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(&S.done)) : "memory");
    __syncwarp();
    for (int it = 0; it < kMaxSpin && !mbar_try_wait(&S.done, 0); ++it) {
    }
  } else if (warp < WARP_BP) {
    // ---- A producers: warp w takes the k-step j = w / 4 of every chunk
    const int q = 32 * (warp & 3) + lane;
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    for (int c = 0; c < nchunk && !*abort; ++c) {
      const int sidx = c % NST;
      {
        DL_T0();
        const bool ok_w = wait_phase(&S.raw_full[sidx], (unsigned)((c / NST) & 1), abort);
        DL_ACC(wt, W_A_RAW_FULL);
        if (!ok_w) break;
      }
      const uint8_t* P = &S.st[sidx].P[q * PBR * 16];
      for (int j = warp >> 2; j < KSC; j += WARP_BP / 4) {
        const int g = c * KSC + j, as = g % GA;
        {
          DL_T0();
          const bool ok_w = g < GA || wait_phase(&S.a_empty[as], (unsigned)(((g / GA) - 1) & 1), abort);
          DL_ACC(wt, W_A_SLOT_EMPTY);
          if (!ok_w) break;
        }
        uint32_t v[2][16];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 pv = *reinterpret_cast<const float4*>(P + (4 * j + r) * 16);
          const float px[2] = {pv.x, pv.z}, py[2] = {pv.y, pv.w};
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float hr = tf32_trunc(px[h]), hi = tf32_trunc(py[h]);
            v[h][2 * r] = __float_as_uint(hr);                      // TF32: k = 2 r + (re, im)
            v[h][2 * r + 1] = __float_as_uint(hi);
            v[h][8 + 2 * r] = pack_bf16(hr, hi);                    // BF16 pair 2 r: hi(P) of row r
            v[h][9 + 2 * r] = pack_bf16(px[h] - hr, py[h] - hi);    // BF16 pair 2 r + 1: lo(P) of row r
          }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
          asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                       "%12, %13, %14, %15, %16};"
                       ::"r"(t_a + 32 * as + 16 * h + lane_off), "r"(v[h][0]), "r"(v[h][1]), "r"(v[h][2]),
                         "r"(v[h][3]), "r"(v[h][4]), "r"(v[h][5]), "r"(v[h][6]), "r"(v[h][7]), "r"(v[h][8]),
                         "r"(v[h][9]), "r"(v[h][10]), "r"(v[h][11]), "r"(v[h][12]), "r"(v[h][13]), "r"(v[h][14]),
                         "r"(v[h][15]) : "memory");
        {
          DL_T0();
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          DL_ACC(wt, W_A_STORE);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.a_full[as]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.raw_empty[sidx]);
    }
  } else if (warp < WARP_MMA) {
    // ---- B producers: warp e (slot e % 2) takes the row pairs e / 2, e / 2
    // + 2, ...; lane (m % 8, row parity, m / 8) writes W_m(y) for
    // y = yc + u_lo + s_row into the columns n = m (Re) and 16 + m (Im) of
    // the row's even block (s_row / 2) and odd block ((s_row - 1) / 2), so
    // that the 16 lanes of a half-warp fill one 128-byte core matrix (8
    // columns n x 2 rows y) per store.  TF32 element (n, row r of the pair
    // starting at row 2 q + par) at q QB + par 512 + (n / 8) 128 + (n % 8) 16
    // + r 8 + (re, im) 4; the BF16 blocks hold per (n, row) four values
    // (hi(P)-part re, im: lo(W); lo(P)-part re, im: W) at r 8 bytes of the
    // same 16-byte column.
    const int e = warp - WARP_BP;
    const int m = 8 * ((lane >> 4) & 1) + (lane & 7), rpar = (lane >> 3) & 1, s = e & 1;
    int am = 0, bm = 0;
    mono_ab(m < NMONO ? m : 0, am, bm);
    const bool live = m < NMONO;
    const int nre = (m / 8) * 128 + (m % 8) * 16, nim = ((16 + m) / 8) * 128 + (m % 8) * 16;
    for (int c = 0; c < nchunk && !*abort; ++c) {
      const int sidx = c % NST, widx = c & 1;   // raw stage, weight-block stage
      {
        DL_T0();
        const bool ok_w = wait_phase(&S.raw_full[sidx], (unsigned)((c / NST) & 1), abort);
        DL_ACC(wt, W_B_RAW_FULL);
        if (!ok_w) break;
      }
      {
        DL_T0();
        const bool ok_w = c < 2 || wait_phase(&S.strip_empty[widx], (unsigned)(((c >> 1) - 1) & 1), abort);
        DL_ACC(wt, W_B_BLK_EMPTY);
        if (!ok_w) break;
      }
      const DStage& st = S.st[sidx];
      const int ybase = Ys + c * CH + ulo;
      uint8_t* tf0 = &S.wblk[widx][s][0][0];
      uint8_t* bf0 = &S.wblk[widx][s][1][0];
#pragma unroll 2
      for (int srow = 2 * (e >> 1) + rpar; srow < VR - 1; srow += 4) {
        const int y = ybase + srow;
        const bool on = live && y >= y0 && y < y1;
        const float2 vv = *reinterpret_cast<const float2*>(&st.V[am][srow * 16 + s * 8]);
        const float yp = st.ypw[srow][2 * bm];
        const float wr = on ? yp * vv.x : 0.f, wi = on ? yp * vv.y : 0.f;
        const float hr = tf32_trunc(wr), hi = tf32_trunc(wi);
        const float lr = wr - hr, li = wi - hi;
        const float2 tre = make_float2(hr, hi), tim = make_float2(-hi, hr);
        const uint2 bre = make_uint2(pack_bf16(lr, li), pack_bf16(wr, wi));
        const uint2 bim = make_uint2(pack_bf16(-li, lr), pack_bf16(-wi, wr));
#pragma unroll
        for (int par = 0; par < 2; ++par) {
          const int rr = srow - par;
          if (rr < 0 || (rr >> 1) >= NQ) continue;
          const int off = (rr >> 1) * QB + (rr & 1) * 8 + par * 512;
          *reinterpret_cast<float2*>(tf0 + nre + off) = tre;
          *reinterpret_cast<float2*>(tf0 + nim + off) = tim;
          *reinterpret_cast<uint2*>(bf0 + nre + off) = bre;
          *reinterpret_cast<uint2*>(bf0 + nim + off) = bim;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&S.strip_full[widx]);
        mbar_arrive(&S.raw_empty[sidx]);
      }
    }
  }

  // ---- drain: the copies of the last NST chunks issued land before the
  // stages are reused (earlier phases of a stage report complete at once)
  if (warp == WARP_COPY)
    for (int c = issued_chunks - NST; c < issued_chunks; ++c) {
      if (c < 0) continue;
      for (int it = 0; it < kMaxSpin && !mbar_try_wait(&S.raw_full[c % NST], (unsigned)((c / NST) & 1)); ++it) {
      }
    }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool ok = nstep > 0 && !S.abort && mbar_try_wait(&S.done, 0);
#ifdef SFFT_DLANE_WAIT_PROFILE
  if (threadIdx.x == 0) wt[W_CTA_CYCLES] = clock64() - cta_t0;
  if (lane == 0)
    for (int k = 0; k < W_NKIND; ++k)
      if (wt[k]) atomicAdd(&g_dl_wait[k], (unsigned long long)wt[k]);
#endif
  if (threadIdx.x == 0 && !ok) atomicOr(reinterpret_cast<int*>(ws + job.status), 4);

  // ---- epilogue: the accumulators of lane q (difference d_first + q) to C[k][d][u_y][32]
  if (ok && warp < 4) {
    const int q = 32 * warp + lane;
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    float* cb = reinterpret_cast<float*>(ws + job.cbuf);
    for (int s = 0; s < 2; ++s)
      for (int i = 0; i < nu; ++i) {
        uint32_t c[32];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                     "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                     "[%32];"
                     : "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7]),
                       "=r"(c[8]), "=r"(c[9]), "=r"(c[10]), "=r"(c[11]), "=r"(c[12]), "=r"(c[13]), "=r"(c[14]),
                       "=r"(c[15]), "=r"(c[16]), "=r"(c[17]), "=r"(c[18]), "=r"(c[19]), "=r"(c[20]), "=r"(c[21]),
                       "=r"(c[22]), "=r"(c[23]), "=r"(c[24]), "=r"(c[25]), "=r"(c[26]), "=r"(c[27]), "=r"(c[28]),
                       "=r"(c[29]), "=r"(c[30]), "=r"(c[31])
                     : "r"(t_d + 32 * (NU * s + i) + lane_off));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (q < job.nlanes) {
          float4* o = reinterpret_cast<float4*>(
              cb + (((int64_t)(k0 + s) * dstride + job.d_first + q) * L + (ulo + i + w)) * 32);
#pragma unroll
          for (int t = 0; t < 8; ++t)
            o[t] = make_float4(__uint_as_float(c[4 * t]), __uint_as_float(c[4 * t + 1]), __uint_as_float(c[4 * t + 2]),
                               __uint_as_float(c[4 * t + 3]));
        }
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(TMEM_COLS) : "memory");
}

template <int DM>
static cudaError_t contract_dlane_dm(const sfft_plan_s* p, int batch_index, int c0, int nc, void* ws) {
  const int job0 = p->dl_first[batch_index], njobs = p->dl_count[batch_index];
  if (njobs <= 0 || nc <= 0) return cudaSuccess;
  const int H = p->d.H, L = p->d.L, B = p->d.batch;
  const size_t smem = sizeof(DSmem);
  auto kern = k_contract_dlane<DM>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int ntot = p->d_batch * p->ccd_group;   // product spectra held: one d-batch of a CCD group
  const int pz = std::min(128, ntot);           // differences per probe box
  // the last tile of a d-batch (93 differences at L = 11) copies a box of its
  // own size rounded up to 8 differences: 27 % fewer copy lines for its CTAs
  const int last_tile = p->d_batch - 128 * ((p->d_batch - 1) / 128);
  const int pzs = std::min(pz, (last_tile + 7) / 8 * 8);
  CUtensorMap mp, mps, mv;
  char* base = static_cast<char*>(ws);
  if (!make_map_blk(&mp, base + p->phat.off, p->M, H, ntot, 4, PBR, pz) ||
      !make_map_blk(&mps, base + p->phat.off, p->M, H, ntot, 4, PBR, pzs) ||
      !make_map(&mv, base + p->wspec.off, p->M, H, p->n_wa * B, 4, VR, 1))
    return cudaErrorInvalidValue;
  const int per_ccd = njobs / B;   // jobs are ordered CCD-major, the same count per CCD
  dim3 grid(per_ccd, p->M / 2, nc);
  kern<<<grid, NTHREADS, smem, p->stream>>>(mp, mps, mv, p->d_dljobs + job0 + (int64_t)c0 * per_ccd, (char*)ws, H, L,
                                            p->d_batch, pz, pzs, (const float*)p->ytab);
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_contract_dlane(const sfft_plan_s* p, int batch_index, int c0, int nc, void* ws) {
  switch (p->DM_KK) {
    case 0: return contract_dlane_dm<0>(p, batch_index, c0, nc, ws);
    case 2: return contract_dlane_dm<2>(p, batch_index, c0, nc, ws);
    case 4: return contract_dlane_dm<4>(p, batch_index, c0, nc, ws);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sfft

extern "C" sfft_status_t sfft_debug_contract_waits(uint64_t* out, int32_t reset) {
#ifdef SFFT_DLANE_WAIT_PROFILE
  if (!out) return SFFT_ERR_ARG;
  unsigned long long h[sfft::W_NKIND];
  if (cudaMemcpyFromSymbol(h, sfft::g_dl_wait, sizeof(h)) != cudaSuccess) return SFFT_ERR_CUDA;
  for (int k = 0; k < sfft::W_NKIND; ++k) out[k] = h[k];
  if (reset) {
    const unsigned long long z[sfft::W_NKIND] = {};
    if (cudaMemcpyToSymbol(sfft::g_dl_wait, z, sizeof(z)) != cudaSuccess) return SFFT_ERR_CUDA;
  }
  return SFFT_OK;
#else
  (void)out;
  (void)reset;
  return SFFT_ERR_UNSUPPORTED;
#endif
}
