// Lag contraction of the product spectra on the fifth-generation tensor cores
// (tcgen05, FP32 path, KK block).
//
// The arithmetic is that of kernels_contract_tc.cu: for one k-slot the y sum
//   C[(d, u_y)][(m, Re|Im)] = sum_y conj(W_m(y)) P^_d(y - u_y),  W_m = yt^b V^_a,
// is a real matrix product whose rows are the (d, u_y) pairs of a pattern (128
// TMEM lanes), whose columns are the monomials (Re: 0..15, Im: 16..31) and whose
// inner dimension runs over rows y and (re, im).  Each product x y is taken as
// hi_x hi_y on the TF32 path (kind::tf32, K = 8 = four rows) plus
// bf16(hi_x) bf16(lo_y) + bf16(lo_x) bf16(y) on the BF16 path (kind::f16,
// K = 16), hi the TF32 truncation and lo = x - hi, as in the split-operand
// scheme of Ootomo and Yokota (2022).  The accumulators of the CTA's eight
// k-slots (32 FP32 columns each) stay in tensor memory for the whole band.
//
// Roles (576 threads, one CTA per SM):
//   warps 0-7  A producers: lane l of warp w is pair 32 (w % 4) + l (warp w
//              reaches tensor-memory lanes 32 (w % 4) ...); per two units
//              (adjacent k-slots, four rows) it loads its probe values from
//              the staged rows (one 16-byte load per row), splits them and
//              stores each unit's 16 A columns to tensor memory (tcgen05.st),
//              warps 0-3 for half of a group's units and warps 4-7 for the
//              other half;
//              warps 0-3 read the accumulators back (tcgen05.ld) at the end for
//              the lag DFT;
//   warps 8-15 B producers: warp 8 + e forms W_m for unit e's four rows and
//              writes its TF32 and BF16 operand tiles (32 x 32 bytes each,
//              K-major, no swizzle) to shared memory, each lane two rows of
//              one monomial with 16- and 8-byte stores;
//   warp 16    MMA issuer: one elected lane issues the sixteen MMAs of a
//              group (two per unit) and one commit;
//   warp 17    copy producer: stages, 32 weight rows at a time and into two
//              alternating stages, one tensor-copy box of probe rows per
//              difference of the pattern, one box of weight rows per exponent
//              and the powers of yt.
// A unit is one k-slot over four rows; a group holds the eight k-slots' units
// of one k-step, and groups alternate between two slots (A: 128 TMEM columns,
// B: 16 KB of shared memory) with mbarrier hand-offs (A written, B written,
// MMAs done), so that one group is built while the tensor cores run the other.
// Every wait is bounded, and a wait that gives up flags the CCD (status bit 4)
// and makes every role leave its loop, after which the issued copies and MMAs
// are drained (bounded) and the tensor memory is freed.
#include <cuda.h>

#include "bulk.cuh"
#include "common.cuh"
#include "plan.h"
#include "umma_common.cuh"

namespace sfft {

namespace {

constexpr int KT = kUmmaKT;          // k-slots per CTA
constexpr int CH = kUmmaChunk;       // weight rows per stage
constexpr int SPG = 1;               // k-steps (four rows each) per group
constexpr int UPG = KT * SPG;        // units (k-slot, k-step) per group
constexpr int GPC = CH / (4 * SPG);  // groups per staged chunk
constexpr int GSLOT = 2;             // groups in flight (A: UPG x 16 TMEM columns, B: UPG x 2 KB each)
constexpr int PITCH = (KT + 2) * 8;  // bytes per staged row: the CTA's KT spectrum slots and 2 more
constexpr int BOXW = PITCH / 4;      // floats per staged row (the tensor box's inner extent)
constexpr int RBOX_MAX = CH + (kMaxL - 1) + 7;   // probe rows per box: chunk, lag range, bank shift
constexpr int DSLOT = (RBOX_MAX * PITCH + 127) / 128 * 128;   // bytes per difference in a stage
constexpr int NDMAX = kUmmaMaxDiffs; // differences per pattern
constexpr int VSLOT = CH * PITCH;    // bytes per weight exponent in a stage
constexpr int WARP_MMA = 16, WARP_COPY = 17;   // warps 0-7: A producers, 8-15: B producers
constexpr int NTHREADS = 32 * 18;
constexpr int TMEM_COLS = 512;       // D: KT x 32 columns, A: GSLOT x UPG x 16 columns
static_assert(KT * 32 + GSLOT * UPG * 16 <= TMEM_COLS, "tensor memory budget");
static_assert(SPG == 1 && KT % 2 == 0 && UPG % 4 == 0, "A producers take two adjacent k-slots per 16-byte load");

// One stage: a box of probe rows per difference (tensor copies; box i starts
// i % 8 rows early so that the differences' rows fall on different banks),
// a box of weight rows per exponent a, and the powers of yt.  Offsets are
// multiples of 128 bytes, as the tensor copies require.
struct UStage {
  uint8_t P[NDMAX][DSLOT];
  uint8_t V[kMaxWeightDeg + 1][VSLOT];
  float ypw[CH][16];
};
static_assert(DSLOT % 128 == 0 && VSLOT % 128 == 0 && sizeof(UStage) % 128 == 0, "tensor copy alignment");

struct USmem {
  UStage st[2];
  uint8_t btile[GSLOT][UPG][2][1024];  // per group slot and unit: TF32 tile, BF16 tile (32 rows x 32 bytes,
                                       // canonical K-major)
  uint64_t raw_full[2], raw_empty[2];
  uint64_t a_full[GSLOT], b_full[GSLOT], mma_done[GSLOT];
  uint64_t done;
  float2 tw[KT][kMaxL];
  uint32_t tmem_base;
  int abort;
};

}  // namespace

template <int DM>
__global__ void __launch_bounds__(NTHREADS, 1)
k_contract_umma(const __grid_constant__ CUtensorMap tmP, const __grid_constant__ CUtensorMap tmV,
                const TcJob* __restrict__ jobs, const int4* __restrict__ pairs, const int4* __restrict__ djobs,
                char* __restrict__ ws, int H, int M, int Nf, int L, int rows_per_cta, int rbox,
                const float2* __restrict__ twD, const float* __restrict__ ytab) {
  constexpr int NMONO = n_mono(DM);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  USmem& S = *reinterpret_cast<USmem*>(smem_raw);
  volatile int* abort = &S.abort;

  const TcJob job = jobs[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int w = (L - 1) / 2;
  const int k0 = blockIdx.x * KT;
  const int4* dj = djobs + job.dj0;
  const int4* pr = pairs + job.pair0;
  int y0 = blockIdx.z * rows_per_cta, y1 = y0 + rows_per_cta;
  if (y0 < w) y0 = w;
  if (y1 > H - w) y1 = H - w;
  const int nchunk = y1 > y0 ? (y1 - y0 + CH - 1) / CH : 0;
  const int ngroup = nchunk * GPC;   // groups of UPG units (k-slot, four rows)
  // ---- setup: zeroed stages, barriers, tensor memory, twiddles
  for (int i = threadIdx.x; i < (int)(sizeof(UStage) * 2 / 16); i += NTHREADS)
    reinterpret_cast<float4*>(&S.st[0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) { mbar_init(&S.raw_full[i], 1); mbar_init(&S.raw_empty[i], 16); }
    for (int i = 0; i < GSLOT; ++i) { mbar_init(&S.a_full[i], 8); mbar_init(&S.b_full[i], 8); mbar_init(&S.mma_done[i], 1); }
    mbar_init(&S.done, 1);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < KT * kMaxL) {
    const int kk = threadIdx.x / kMaxL, ux = threadIdx.x % kMaxL - w;
    int idx = (int)(((int64_t)(k0 + kk) * ux) % Nf);
    if (idx < 0) idx += Nf;
    const float2 cs = twD[idx];
    S.tw[kk][threadIdx.x % kMaxL] = make_float2(2.f * cs.x, 2.f * cs.y);
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
  const uint32_t t_d = tbase;                   // accumulators: k-slot kk at columns 32 kk
  const uint32_t t_a = tbase + 32 * KT;         // A: group slot g, unit e at columns 16 (UPG g + e)
                                                // (TF32 0-7, BF16 8-15)

  int issued_chunks = 0;   // bulk-copy warp: chunks whose copies were issued

  if (warp == WARP_COPY) {
    // ---- copy producer: per chunk one tensor copy per difference and per
    // weight exponent and one bulk copy of the powers of yt
    for (int c = 0; c < nchunk; ++c) {
      const int sidx = c & 1;
      if (c >= 2 && !wait_phase(&S.raw_empty[sidx], (unsigned)(((c >> 1) - 1) & 1), abort)) break;
      UStage& st = S.st[sidx];
      const int yc = y0 + c * CH, ye = min(yc + CH, y1), nrow = ye - yc;
      if (lane == 0)
        mbar_arrive_expect_tx(&S.raw_full[sidx], (unsigned)(job.nd * rbox * PITCH + (DM + 1) * VSLOT + nrow * 64));
      __syncwarp();
      if (lane < job.nd) {
        const int4 e = dj[lane];   // (d_local, u_lo, u_hi, -): rows yc - u_hi - lane % 8 ...
        tma_load_3d(&st.P[lane][0], &tmP, 2 * k0, yc - e.z - lane % 8, job.zp + e.x, &S.raw_full[sidx]);
      } else if (lane < job.nd + DM + 1) {
        const int a = lane - job.nd;
        tma_load_3d(&st.V[a][0], &tmV, 2 * k0, yc, job.zw + a, &S.raw_full[sidx]);
      } else if (lane == 31) {
        bulk_copy_g2s(&st.ypw[0][0], ytab + (int64_t)yc * 16, (unsigned)(nrow * 64), &S.raw_full[sidx]);
      }
      issued_chunks = c + 1;
      __syncwarp();
    }
  } else if (warp == WARP_MMA) {
    // ---- MMA issuer: per group, two MMAs per unit and one commit
    constexpr uint32_t id_tf32 = instr_desc(2), id_bf16 = instr_desc(1);
    for (int g = 0; g < ngroup; ++g) {
      const int slot = g % GSLOT;
      const unsigned par = (unsigned)((g / GSLOT) & 1);
      if (!wait_phase(&S.a_full[slot], par, abort) || !wait_phase(&S.b_full[slot], par, abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (elect_one()) {
#pragma unroll
        for (int e = 0; e < UPG; ++e) {   // unit e: k-slot e / SPG, k-step e % SPG of the group
          const int kk = e / SPG;
          const uint32_t acc = (g > 0 || e % SPG > 0) ? 1u : 0u;   // the first k-step starts the accumulators
          const uint32_t dcol = t_d + 32 * kk, acol = t_a + 16 * (UPG * slot + e);
          const uint64_t bt = smem_desc(smem_u32(&S.btile[slot][e][0][0]));
          const uint64_t bb = smem_desc(smem_u32(&S.btile[slot][e][1][0]));
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                       ::"r"(dcol), "r"(acol), "l"(bt), "r"(id_tf32), "r"(acc) : "memory");
          asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                       " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n"
                       ::"r"(dcol), "r"(acol + 8), "l"(bb), "r"(id_bf16), "r"(1u) : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&S.mma_done[slot])) : "memory");
      }
      __syncwarp();
    }
    // every MMA issued so far completes before the accumulators are read or freed
    if (elect_one())
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   ::"r"(smem_u32(&S.done)) : "memory");
    __syncwarp();
    for (int it = 0; it < kMaxSpin && !mbar_try_wait(&S.done, 0); ++it) {
    }
  } else if (warp < 8) {
    // ---- A producers: lanes of warp w hold pair q = 32 (w % 4) + lane (their
    // tensor-memory lanes); warp w writes units UPG / 2 (w / 4) ... of every
    // group, then waits for its stores once and arrives
    const int quarter = warp & 3, e0 = (UPG / 2) * (warp >> 2);
    int q = 32 * quarter + lane;
    if (q >= job.npair) q = 0;   // lanes past the pattern mirror pair 0; their rows are dropped
    const int4 pq = pr[q];
    int off0 = 0;   // byte offset in a stage of (pair, weight row yc, slot 0)
    for (int i = 0; i < job.nd; ++i)
      if (dj[i].x == pq.x) off0 = i * DSLOT + (dj[i].z + i % 8 - pq.y) * PITCH;
    const uint32_t lane_off = (uint32_t)(32 * quarter) << 16;
    for (int c = 0; c < nchunk && !*abort; ++c) {
      const int sidx = c & 1;
      if (!wait_phase(&S.raw_full[sidx], (unsigned)((c >> 1) & 1), abort)) break;
      const uint8_t* P = &S.st[sidx].P[0][0] + off0;
      for (int sp = 0; sp < GPC; ++sp) {
        const int g = c * GPC + sp, slot = g % GSLOT;
        if (g >= GSLOT && !wait_phase(&S.mma_done[slot], (unsigned)(((g / GSLOT) - 1) & 1), abort)) break;
#pragma unroll
        for (int e = e0; e < e0 + UPG / 2; e += 2) {   // units e, e + 1: adjacent k-slots, one 16-byte load per row
          const int kk = e, s = sp;
          uint32_t v[2][16];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float4 pv = *reinterpret_cast<const float4*>(P + (4 * s + r) * PITCH + kk * 8);
            const float px[2] = {pv.x, pv.z}, py[2] = {pv.y, pv.w};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float hr = tf32_trunc(px[h]), hi = tf32_trunc(py[h]);
              v[h][2 * r] = __float_as_uint(hr);        // TF32 columns: k = 2 r + (re, im)
              v[h][2 * r + 1] = __float_as_uint(hi);
              v[h][8 + r] = pack_bf16(hr, hi);          // BF16 columns 0-3: hi(P) of row r
              v[h][12 + r] = pack_bf16(px[h] - hr, py[h] - hi);   // BF16 columns 4-7: lo(P) of row r
            }
          }
#pragma unroll
          for (int h = 0; h < 2; ++h)
            asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                         "%12, %13, %14, %15, %16};"
                         ::"r"(t_a + 16 * (UPG * slot + e + h) + lane_off), "r"(v[h][0]), "r"(v[h][1]), "r"(v[h][2]),
                           "r"(v[h][3]), "r"(v[h][4]), "r"(v[h][5]), "r"(v[h][6]), "r"(v[h][7]), "r"(v[h][8]),
                           "r"(v[h][9]), "r"(v[h][10]), "r"(v[h][11]), "r"(v[h][12]), "r"(v[h][13]), "r"(v[h][14]),
                           "r"(v[h][15]) : "memory");
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.a_full[slot]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.raw_empty[sidx]);
    }
  } else {
    // ---- B producers: warp 8 + e builds the tiles of unit e (k-slot e / SPG,
    // k-step e % SPG) of every group; lane: monomial m = lane % 16, rows
    // r = lane / 16 and + 2
    const int e = warp - 8, kk = e / SPG;
    const int m = lane & 15, rp = lane >> 4;
    int am = 0, bm = 0;
    mono_ab(m < NMONO ? m : 0, am, bm);
    const bool live = m < NMONO;
    for (int c = 0; c < nchunk && !*abort; ++c) {
      const int sidx = c & 1;
      if (!wait_phase(&S.raw_full[sidx], (unsigned)((c >> 1) & 1), abort)) break;
      const UStage& st = S.st[sidx];
      const int yc = y0 + c * CH, ye = min(yc + CH, y1);
      for (int sp = 0; sp < GPC; ++sp) {
        const int g = c * GPC + sp, slot = g % GSLOT, s = SPG * sp + e % SPG;
        if (g >= GSLOT && !wait_phase(&S.mma_done[slot], (unsigned)(((g / GSLOT) - 1) & 1), abort)) break;
        {
          uint8_t* tf = &S.btile[slot][e][0][0];
          uint8_t* tb = &S.btile[slot][e][1][0];
          float wr[2], wi[2], hr[2], hi[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int row = 4 * s + 2 * rp + h;
            const bool on = live && yc + row < ye;
            const float2 vv = *reinterpret_cast<const float2*>(&st.V[am][row * PITCH + kk * 8]);
            const float yp = st.ypw[row][2 * bm];
            wr[h] = on ? yp * vv.x : 0.f;
            wi[h] = on ? yp * vv.y : 0.f;
            hr[h] = tf32_trunc(wr[h]);
            hi[h] = tf32_trunc(wi[h]);
          }
          // rows n = m (Re) and 16 + m (Im); element (n, k) of the TF32 tile at
          // (n / 8) 256 + (k / 4) 128 + (n % 8) 16 + (k % 4) 4, k = 2 r + (re, im):
          // this lane's rows 2 rp, 2 rp + 1 fill one 16-byte core-matrix row
          const int nre = (m / 8) * 256 + (m % 8) * 16, nim = ((16 + m) / 8) * 256 + (m % 8) * 16;
          *reinterpret_cast<float4*>(tf + nre + rp * 128) = make_float4(hr[0], hi[0], hr[1], hi[1]);
          *reinterpret_cast<float4*>(tf + nim + rp * 128) = make_float4(-hi[0], hr[0], -hi[1], hr[1]);
          // BF16 tile: element (n, k) at (n / 8) 256 + (k / 8) 128 + (n % 8) 16 + (k % 8) 2;
          // k = 2 r + (re, im) multiplies hi(P), k = 8 + 2 r + (re, im) multiplies lo(P)
          const float lr0 = wr[0] - hr[0], li0 = wi[0] - hi[0], lr1 = wr[1] - hr[1], li1 = wi[1] - hi[1];
          const int kb1 = rp * 8;
          *reinterpret_cast<uint2*>(tb + nre + kb1) = make_uint2(pack_bf16(lr0, li0), pack_bf16(lr1, li1));
          *reinterpret_cast<uint2*>(tb + nim + kb1) = make_uint2(pack_bf16(-li0, lr0), pack_bf16(-li1, lr1));
          *reinterpret_cast<uint2*>(tb + nre + 128 + kb1) =
              make_uint2(pack_bf16(wr[0], wi[0]), pack_bf16(wr[1], wi[1]));
          *reinterpret_cast<uint2*>(tb + nim + 128 + kb1) =
              make_uint2(pack_bf16(-wi[0], wr[0]), pack_bf16(-wi[1], wr[1]));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.b_full[slot]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&S.raw_empty[sidx]);
    }
  }

  // ---- drain: the copies of the last two chunks issued land before the
  // stages are reused (earlier phases of a stage report complete at once)
  if (warp == WARP_COPY)
    for (int c = issued_chunks - 2; c < issued_chunks; ++c) {
      if (c < 0) continue;
      for (int it = 0; it < kMaxSpin && !mbar_try_wait(&S.raw_full[c & 1], (unsigned)((c >> 1) & 1)); ++it) {
      }
    }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool ok = ngroup > 0 && !S.abort && mbar_try_wait(&S.done, 0);
  if (threadIdx.x == 0 && !ok) atomicOr(reinterpret_cast<int*>(ws + job.status), 4);

  // ---- epilogue: lag DFT over the CTA's k-slots, per pair in thread-private
  // shared sums (fixed order), then FP64 atomics
  constexpr int RSTRIDE = 16 * kMaxL + 1;
  float* red = reinterpret_cast<float*>(&S.st[0]);   // [128][RSTRIDE], aliases the stages
  if (ok && warp < 4) {
    const int q = 32 * warp + lane;
    const int4 pq = pr[q < job.npair ? q : 0];
    float* rq = red + q * RSTRIDE;
    for (int i = 0; i < 16 * kMaxL; ++i) rq[i] = 0.f;
    const uint32_t lane_off = (uint32_t)(32 * warp) << 16;
    for (int kk = 0; kk < KT; ++kk) {
      uint32_t c[32];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                   "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                   "[%32];"
                   : "=r"(c[0]), "=r"(c[1]), "=r"(c[2]), "=r"(c[3]), "=r"(c[4]), "=r"(c[5]), "=r"(c[6]), "=r"(c[7]),
                     "=r"(c[8]), "=r"(c[9]), "=r"(c[10]), "=r"(c[11]), "=r"(c[12]), "=r"(c[13]), "=r"(c[14]),
                     "=r"(c[15]), "=r"(c[16]), "=r"(c[17]), "=r"(c[18]), "=r"(c[19]), "=r"(c[20]), "=r"(c[21]),
                     "=r"(c[22]), "=r"(c[23]), "=r"(c[24]), "=r"(c[25]), "=r"(c[26]), "=r"(c[27]), "=r"(c[28]),
                     "=r"(c[29]), "=r"(c[30]), "=r"(c[31])
                   : "r"(t_d + 32 * kk + lane_off));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int k = k0 + kk;
      if (k == 0 || k >= M) continue;   // slot 0: the packed real bins, summed by k_contract_slot0
      for (int ux = pq.z; ux <= pq.w; ++ux) {
        const float2 t2 = S.tw[kk][ux + w];
#pragma unroll
        for (int mm = 0; mm < NMONO; ++mm)
          rq[mm * kMaxL + ux + w] += __uint_as_float(c[mm]) * t2.x + __uint_as_float(c[16 + mm]) * t2.y;
      }
    }
    if (q < job.npair) {
      const double inv = 1.0 / (double)Nf;
      double* out = reinterpret_cast<double*>(ws + job.out) + ((int64_t)pq.x * L * L + (pq.y + w) * L) * NMONO;
      for (int ux = pq.z; ux <= pq.w; ++ux)
#pragma unroll
        for (int mm = 0; mm < NMONO; ++mm) {
          const float v = rq[mm * kMaxL + ux + w];
          if (v != 0.f) atomicAdd(out + (ux + w) * NMONO + mm, (double)v * inv);
        }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(TMEM_COLS) : "memory");
}

template <int DM>
static cudaError_t contract_umma_dm(const sfft_plan_s* p, int job0, int njobs, void* ws) {
  const size_t smem = sizeof(USmem);
  static_assert(sizeof(float) * 128 * (16 * kMaxL + 1) <= 2 * sizeof(UStage), "epilogue sums must fit the stages");
  auto kern = k_contract_umma<DM>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int H = p->d.H, L = p->d.L, B = p->d.batch;
  const int rows = p->tc_rows;
  const int nb = (H + rows - 1) / rows;
  const int rbox = CH + (L - 1) + 7;
  // one launch for every CCD of the batch: the product and weight spectra of
  // all CCDs are consecutive slabs, so one tensor map covers each kind and a
  // job names its CCD's first slab
  CUtensorMap mp, mv;
  char* base = static_cast<char*>(ws);
  if (!make_map(&mp, base + p->phat.off, p->M, H, p->d_batch * p->ccd_group, BOXW, rbox, 1) ||
      !make_map(&mv, base + p->wspec.off, p->M, H, p->n_wa * B, BOXW, CH, 1))
    return cudaErrorInvalidValue;
  for (int j0 = 0; j0 < njobs; j0 += 65535) {
    dim3 grid(p->M / KT, std::min(65535, njobs - j0), nb);
    kern<<<grid, NTHREADS, smem, p->stream>>>(mp, mv, p->d_tcjobs + job0 + j0, p->d_tcpairs, p->d_tcdj, (char*)ws, H,
                                              p->M, p->Nf, L, rows, rbox, (const float2*)p->twD,
                                              (const float*)p->ytab);
    p->nlaunch += 1;
  }
  return cudaGetLastError();
}

cudaError_t launch_contract_umma(const sfft_plan_s* p, int batch_index, int c0, int nc, void* ws) {
  // jobs are ordered CCD-major with the same count per CCD: the group's jobs are one run
  const int per_ccd = p->tc_count[batch_index] / p->d.batch;
  const int job0 = p->tc_first[batch_index] + c0 * per_ccd, njobs = nc * per_ccd;
  if (njobs <= 0) return cudaSuccess;
  switch (p->DM_KK) {
    case 0: return contract_umma_dm<0>(p, job0, njobs, ws);
    case 2: return contract_umma_dm<2>(p, job0, njobs, ws);
    case 4: return contract_umma_dm<4>(p, job0, njobs, ws);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sfft
