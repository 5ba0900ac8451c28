// Batched real-to-complex row FFTs with shared-memory staging.
//
// Row length Nf = 2M (power of two, 64..2048, zero padded past W).  The real
// row x[n] is packed as z[n] = x[2n] + i x[2n+1] (M points) and transformed by
// an autosorting (Stockham) radix-16 decomposition: M = 16 * 16 * ... * R_last,
// each pass a length-R DFT in registers over inputs M/R apart, with twiddles
// exp(-2 pi i r k / (Ns R)) where Ns is the product of the earlier radices and
// k = j mod Ns.  A row is handled by M/16 threads that each hold 16 complex
// values; the rows of a CTA move through the passes in lockstep and exchange
// data in padded shared memory (one pad word per 16 keeps the strided pass
// accesses free of bank conflicts).  The final split gives the real-input
// spectrum X[k], k = 0..M.  Output row layout: M complex slots, slot 0 packs
// the two real bins (X[0], X[M]); slot k holds X[k] otherwise.
//
// Three row sources feed the same transform:
//   products   P_d(y, x) = R_m(y, x) R_m(y + d_y, x + d_x)   (zero off-image)
//   reference  R_m(y, x)
//   weights    M_fit(y, x) xt^a [ * (S(y, x) - s_S) | * e(y, x) ]
#include "common.cuh"
#include "plan.h"

namespace sfft {

constexpr int kFftThreads = 256;

__host__ __device__ constexpr int fft_pad(int i) { return i + (i >> 4); }

template <typename T, int M>
struct RowFFT {
  using T2 = c_t<T>;
  static constexpr int TPR = M / 16;              // threads per row
  static constexpr int RPB = kFftThreads / TPR;   // rows per CTA
  static constexpr int SROW = fft_pad(M) + 1;     // padded complex elements per row
  static constexpr size_t smem_bytes() { return sizeof(T2) * (size_t)SROW * RPB; }

  // One Stockham pass of radix R with span NS over shared memory (in place:
  // every thread loads its inputs, the CTA synchronizes, then stores).
  template <int R, int NS>
  __device__ static void pass(T2* buf, int t, const T2* __restrict__ tw) {
    constexpr int Q = 16 / R;
    T2 v[Q][R];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int j = t + TPR * q;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = buf[fft_pad(j + r * (M / R))];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int j = t + TPR * q;
      const int k = j % NS;
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], tw[r * k * (M / (NS * R))]);
      }
      fft_reg<R>(v[q]);
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[fft_pad(base + r * NS)] = v[q][r];
    }
    __syncthreads();
  }

  template <int NS>
  __device__ static void passes(T2* buf, int t, const T2* tw) {
    if constexpr (NS < M) {
      constexpr int R = (M / NS) >= 16 ? 16 : (M / NS);
      pass<R, NS>(buf, t, tw);
      passes<NS * R>(buf, t, tw);
    }
  }

  // v[r] = z[t + TPR r] (the first pass's inputs, radix 16, span 1) -> spectrum row `out`
  // (X[k] is stored at out[k], or with BLK at out[(k / 16) kb + k % 16] for
  // the k-slot-blocked product spectra, kb = 16 H)
  template <bool BLK = false>
  __device__ static void run(T2 (&v)[16], T2* buf, int t, bool valid, const T2* __restrict__ twM,
                             const T2* __restrict__ twN, T2* __restrict__ out, int kb = 0) {
    // first pass straight from registers
    fft_reg<16>(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[fft_pad(t * 16 + r)] = v[r];
    __syncthreads();
    passes<16>(buf, t, twM);
    // real-input split: X[k] = E + (-i) exp(-2 pi i k / Nf) O
    if (valid) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int k = t + TPR * q;
        const int km = (M - k) & (M - 1);
        const T2 zk = buf[fft_pad(k)], zm = buf[fft_pad(km)];
        T2 X;
        if (k == 0) {
          X.x = zk.x + zk.y;
          X.y = zk.x - zk.y;
        } else {
          const T er = (T)0.5 * (zk.x + zm.x), ei = (T)0.5 * (zk.y - zm.y);
          const T orr = (T)0.5 * (zk.x - zm.x), oi = (T)0.5 * (zk.y + zm.y);
          const T2 wk = twN[k];
          const T wr = wk.x * orr - wk.y * oi, wi = wk.x * oi + wk.y * orr;
          X.x = er + wi;
          X.y = ei - wr;
        }
        if constexpr (BLK) out[(k >> 4) * kb + (k & 15)] = X;
        else out[k] = X;
      }
    }
    __syncthreads();
  }
};

// products (self == 0) or the plain R_m spectrum (self == 1)
template <typename T, int M>
__global__ void __launch_bounds__(kFftThreads)
k_rfft_prod(const T* __restrict__ Rm, int H, int W, const int2* __restrict__ dl, int d0, int self,
            c_t<T>* __restrict__ out, int64_t slab_stride, int64_t ccd_stride_out,
            const c_t<T>* __restrict__ twM, const c_t<T>* __restrict__ twN) {
  using F = RowFFT<T, M>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rloc = threadIdx.x / F::TPR, t = threadIdx.x % F::TPR;
  c_t<T>* buf = reinterpret_cast<c_t<T>*>(smem_raw) + (size_t)rloc * F::SROW;
  const int jd = blockIdx.y, ccd = blockIdx.z;
  int dy = 0, dx = 0;
  if (!self) { const int2 dd = dl[d0 + jd]; dy = dd.x; dx = dd.y; }
  const T* img = Rm + (int64_t)ccd * H * W;
  c_t<T>* obase = out + (int64_t)ccd * ccd_stride_out + (int64_t)jd * slab_stride;
  for (int yb = blockIdx.x * F::RPB; yb < H; yb += gridDim.x * F::RPB) {
    const int y = yb + rloc;
    const bool valid = y < H;
    const bool ok2 = valid && (y + dy >= 0) && (y + dy < H);
    const T* row = img + (int64_t)(valid ? y : 0) * W;
    const T* row2 = img + (int64_t)(ok2 ? y + dy : 0) * W;
    c_t<T> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int x0 = 2 * (t + F::TPR * r), x1 = x0 + 1;
      T v0 = (valid && x0 < W) ? row[x0] : (T)0;
      T v1 = (valid && x1 < W) ? row[x1] : (T)0;
      if (!self) {
        const int s0 = x0 + dx, s1 = x1 + dx;
        v0 *= (ok2 && s0 >= 0 && s0 < W) ? row2[s0] : (T)0;
        v1 *= (ok2 && s1 >= 0 && s1 < W) ? row2[s1] : (T)0;
      }
      v[r].x = v0;
      v[r].y = v1;
    }
    F::run(v, buf, t, valid, twM, twN, obase + (int64_t)(valid ? y : 0) * M);
  }
}

// Products for one image row y and one kernel-offset row difference d_y: the
// CTA stages R_m(y, .) and R_m(y + d_y, .) in shared memory (zero padded by
// 16 on each side for the d_x shift), then forms RPB products at a time -- one
// per d_x of this d_y in the batch -- and transforms them side by side.
// grid = (H, number of d_y values met by the batch [d0, d0 + nd), batch).
template <typename T, int M, bool BLK>
__global__ void __launch_bounds__(kFftThreads)
k_rfft_prod_dy(const T* __restrict__ Rm, int H, int W, int L, int d0, int nd, c_t<T>* __restrict__ out,
               int64_t slab_stride, int64_t ccd_stride_out, const c_t<T>* __restrict__ twM,
               const c_t<T>* __restrict__ twN) {
  using F = RowFFT<T, M>;
  constexpr int NF = 2 * M, PADX = 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  c_t<T>* bufs = reinterpret_cast<c_t<T>*>(smem_raw);
  T* r1 = reinterpret_cast<T*>(smem_raw + F::smem_bytes());   // [NF]
  T* r2 = r1 + NF;                                              // [NF + 2 PADX]
  const int rloc = threadIdx.x / F::TPR, t = threadIdx.x % F::TPR;
  c_t<T>* buf = bufs + (size_t)rloc * F::SROW;
  const int y = blockIdx.x, ccd = blockIdx.z;
  // half-plane order: d_y = 0 holds d_x = 0..L-1, each d_y > 0 holds d_x = -(L-1)..L-1
  auto first_of = [L](int dy) { return dy == 0 ? 0 : L + (2 * L - 1) * (dy - 1); };
  auto dy_of = [L](int id) { return id < L ? 0 : 1 + (id - L) / (2 * L - 1); };
  const int dy = dy_of(d0) + blockIdx.y;
  const int lo = max(d0, first_of(dy)), hi = min(d0 + nd, first_of(dy) + (dy == 0 ? L : 2 * L - 1));
  if (lo >= hi) return;   // uniform over the CTA
  const T* img = Rm + (int64_t)ccd * H * W;
  const bool ok2 = y + dy < H;
  for (int x = threadIdx.x; x < NF; x += blockDim.x) r1[x] = x < W ? img[(int64_t)y * W + x] : (T)0;
  for (int x = threadIdx.x; x < NF + 2 * PADX; x += blockDim.x) {
    const int gx = x - PADX;
    r2[x] = (ok2 && gx >= 0 && gx < W) ? img[(int64_t)(y + dy) * W + gx] : (T)0;
  }
  __syncthreads();
  const int dx0 = dy == 0 ? 0 : -(L - 1);
  c_t<T>* obase = out + (int64_t)ccd * ccd_stride_out + (int64_t)y * (BLK ? 16 : M);
  for (int id0 = lo; id0 < hi; id0 += F::RPB) {
    const int id = id0 + rloc;
    const bool valid = id < hi;
    const int dx = dx0 + (id - first_of(dy));
    c_t<T> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int x0 = 2 * (t + F::TPR * r);
      // products vanish where R_m(y + d_y, x + d_x) falls outside the image (r2 is zero there)
      v[r].x = valid ? r1[x0] * r2[x0 + dx + PADX] : (T)0;
      v[r].y = valid ? r1[x0 + 1] * r2[x0 + 1 + dx + PADX] : (T)0;
    }
    F::template run<BLK>(v, buf, t, valid, twM, twN, obase + (int64_t)(valid ? id - d0 : 0) * slab_stride, 16 * H);
  }
}

// FP32 products for 2048-sample rows (M = 1024), one warp per product row.
// Four-step transform of the packed row z[n], n = l + 32 q (lane l holds the
// 32 samples q): a 32-point DFT over q in registers, the twiddle
// exp(-2 pi i l a / 1024), a transpose through the warp's own shared-memory
// tile, and a 32-point DFT over l, after which lane a holds X[a + 32 b].  The
// real-input split reads X[M - k] back from the same tile.  Only warp-level
// synchronisation is needed between the staged source rows and the output.
// Each CTA walks `rows` image rows of one d_y group; its 8 warps take the
// d_x values of the group in turns.
constexpr int kWarpRowsPerCta = 4;

// The rest of a 2048-sample real row transform for one warp: v[q] holds the
// packed samples z[lane + 32 q]; the spectrum X[k], k = 0 .. 1023 (slot 0: the
// two real bins), goes to o[k], or with BLK to o[(k / 16) 16 H + k % 16].
// Twiddles of the 2048-sample row transform for lane l: mid(a) =
// exp(-2 pi i l a / 1024) between the two 32-point passes, split(b) =
// exp(-2 pi i (l + 32 b) / 2048) for the real-input split, formed from 13
// per-lane values (mid(a) = tB[a mod 8] tA[a / 8]).  (Read from a table in
// shared memory instead they measured slower: 2.60 against 2.49 ms for the
// product FFTs of the DECam pair.)
struct TwReg {
  float2 tB[8], tA[4], tn;
  __device__ __forceinline__ void load(const float2* __restrict__ twM, const float2* __restrict__ twN) {
    constexpr int M = 1024;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = 0; i < 8; ++i) tB[i] = twM[(lane * i) & (M - 1)];
#pragma unroll
    for (int j = 0; j < 4; ++j) tA[j] = twM[(8 * lane * j) & (M - 1)];
    tn = twN[lane];
  }
  __device__ __forceinline__ float2 mid(int a) const {
    float2 w = tB[a & 7];
    if ((a >> 3) != 0) w = (a & 7) ? cmul(w, tA[a >> 3]) : tA[a >> 3];
    return w;
  }
  __device__ __forceinline__ float2 split(int b) const { return twiddle_mul(tn, b, 64); }
};

template <bool BLK, typename TW>
__device__ __forceinline__ void warp_rfft2048_finish(float2 (&v)[32], float2* tile, const TW& tw,
                                                     float2* __restrict__ o, int H) {
  constexpr int M = 1024, SROW = 33;
  const int lane = threadIdx.x & 31;
  fft_reg<32>(v);   // over q: v[a]
#pragma unroll
  for (int a = 1; a < 32; ++a) v[a] = cmul(v[a], tw.mid(a));
#pragma unroll
  for (int a = 0; a < 32; ++a) tile[lane * SROW + a] = v[a];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = tile[j * SROW + lane];
  __syncwarp();
  fft_reg<32>(v);   // over l: v[b] = X[lane + 32 b]
#pragma unroll
  for (int b = 0; b < 32; ++b) tile[lane + 32 * b] = v[b];
  __syncwarp();
  // the real-input split in pairs (k, M - k): lane l takes k = l + 32 b,
  // b < 16, and M - k (lane 32 - l's upper half; lanes 0 and 16 pair with
  // themselves), so both outputs share the sums, the differences and the
  // twiddle w_k (w_{M-k} = -conj(w_k)); lane 0 also takes k = M / 2
  auto put = [&](int k, float2 X) {
    if constexpr (BLK) o[(int64_t)(k >> 4) * (16 * H) + (k & 15)] = X;   // [k / 16][y][k % 16]
    else o[k] = X;
  };
#pragma unroll
  for (int b = 0; b < 16; ++b) {
    const int k = lane + 32 * b;
    const float2 zk = v[b], zm = tile[(M - k) & (M - 1)];
    const float er = 0.5f * (zk.x + zm.x), ei = 0.5f * (zk.y - zm.y);
    const float orr = 0.5f * (zk.x - zm.x), oi = 0.5f * (zk.y + zm.y);
    const float2 wk = tw.split(b);   // exp(-2 pi i (lane + 32 b) / NF)
    const float wr = wk.x * orr - wk.y * oi, wi = wk.x * oi + wk.y * orr;
    if (b == 0 && lane == 0) {
      put(0, make_float2(zk.x + zk.y, zk.x - zk.y));   // slot 0: the two real bins
    } else {
      put(k, make_float2(er + wi, ei - wr));
      put(M - k, make_float2(er - wi, -ei - wr));
    }
  }
  if (lane == 0) {   // k = M / 2 pairs with itself
    const float2 z = v[16];
    const float2 wk = tw.split(16);
    const float wr = -wk.y * z.y, wi = wk.x * z.y;   // orr = 0, oi = z.y
    put(M / 2, make_float2(z.x + wi, -wr));
  }
}



template <bool BLK>
__global__ void __launch_bounds__(256, 2)
k_rfft_prod_dy_w(const float* __restrict__ Rm, int H, int W, int L, int d0, int nd, float2* __restrict__ out,
                 int64_t slab_stride, int64_t ccd_stride_out, const float2* __restrict__ twM,
                 const float2* __restrict__ twN) {
  constexpr int M = 1024, NF = 2048, PADX = 16, SROW = 33;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* r1 = reinterpret_cast<float*>(smem_raw);            // [NF]
  float* r2 = r1 + NF;                                         // [NF + 2 PADX]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* tile = reinterpret_cast<float2*>(r2 + NF + 2 * PADX) + warp * 32 * SROW;
  TwReg tw;
  tw.load(twM, twN);
  const int ccd = blockIdx.z;
  auto first_of = [L](int dy) { return dy == 0 ? 0 : L + (2 * L - 1) * (dy - 1); };
  auto dy_of = [L](int id) { return id < L ? 0 : 1 + (id - L) / (2 * L - 1); };
  const int dy = dy_of(d0) + blockIdx.y;
  const int lo = max(d0, first_of(dy)), hi = min(d0 + nd, first_of(dy) + (dy == 0 ? L : 2 * L - 1));
  if (lo >= hi) return;   // uniform over the CTA
  const int dx0 = dy == 0 ? 0 : -(L - 1);
  const float* img = Rm + (int64_t)ccd * H * W;
  for (int yy = 0; yy < kWarpRowsPerCta; ++yy) {
    const int y = blockIdx.x * kWarpRowsPerCta + yy;
    if (y >= H) break;   // uniform
    __syncthreads();     // the previous row's products are formed
    const bool ok2 = y + dy < H;
    for (int x = threadIdx.x; x < NF; x += blockDim.x) r1[x] = x < W ? img[(int64_t)y * W + x] : 0.f;
    for (int x = threadIdx.x; x < NF + 2 * PADX; x += blockDim.x) {
      const int gx = x - PADX;
      r2[x] = (ok2 && gx >= 0 && gx < W) ? img[(int64_t)(y + dy) * W + gx] : 0.f;
    }
    __syncthreads();
    float2* orow = out + (int64_t)ccd * ccd_stride_out + (int64_t)y * (BLK ? 16 : M);
    for (int id = lo + warp; id < hi; id += 8) {
      const int dx = dx0 + (id - first_of(dy));
      float2 v[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int x0 = 2 * (lane + 32 * q);
        const float2 a = *reinterpret_cast<const float2*>(r1 + x0);
        // products vanish where R_m(y + d_y, x + d_x) falls outside the image (r2 is zero there)
        v[q].x = a.x * r2[x0 + dx + PADX];
        v[q].y = a.y * r2[x0 + 1 + dx + PADX];
      }
      warp_rfft2048_finish<BLK>(v, tile, tw, orow + (int64_t)(id - d0) * slab_stride, H);
      __syncwarp();
    }
  }
}

// weights M_fit xt^a, optionally times (S - s_S) (S != null) or e (E != null)
template <typename T, int M>
__global__ void __launch_bounds__(kFftThreads)
k_rfft_weight(const uint8_t* __restrict__ Mfit, const float* __restrict__ S, const double* __restrict__ sky,
              const T* __restrict__ E, int H, int W, int a0, c_t<T>* __restrict__ out, int64_t slab_stride,
              int64_t ccd_stride_out, const c_t<T>* __restrict__ twM, const c_t<T>* __restrict__ twN) {
  using F = RowFFT<T, M>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int rloc = threadIdx.x / F::TPR, t = threadIdx.x % F::TPR;
  c_t<T>* buf = reinterpret_cast<c_t<T>*>(smem_raw) + (size_t)rloc * F::SROW;
  const int a = a0 + blockIdx.y, ccd = blockIdx.z;
  const int64_t img_off = (int64_t)ccd * H * W;
  const T sS = S ? (T)sky[2 * ccd + 1] : (T)0;
  const T xs = (T)2.0 / (T)(W > 1 ? W - 1 : 1);
  c_t<T>* obase = out + (int64_t)ccd * ccd_stride_out + (int64_t)blockIdx.y * slab_stride;
  for (int yb = blockIdx.x * F::RPB; yb < H; yb += gridDim.x * F::RPB) {
    const int y = yb + rloc;
    const bool valid = y < H;
    const int64_t roff = img_off + (int64_t)(valid ? y : 0) * W;
    c_t<T> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      T vv[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int x = 2 * (t + F::TPR * r) + h;
        T val = (T)0;
        if (valid && x < W && Mfit[roff + x]) {
          const T xt = (T)x * xs - (T)1;
          T pw = (T)1;
          for (int i = 0; i < a; ++i) pw *= xt;
          if (S) pw *= ((T)S[roff + x] - sS);
          else if (E) pw *= E[roff + x];
          val = pw;
        }
        vv[h] = val;
      }
      v[r].x = vv[0];
      v[r].y = vv[1];
    }
    F::run(v, buf, t, valid, twM, twN, obase + (int64_t)(valid ? y : 0) * M);
  }
}

// FP32 weight spectra of 2048-sample rows (M = 1024) with the transform of
// k_rfft_prod_dy_w.  A CTA walks kWarpRowsPerCta rows; per row it stages the
// samples f(x) xt^a, f(x) = M_fit(x) [ (S(x) - s_S) | e(x) | 1 ], of all
// na <= kMaxWeightDeg + 1 spectra in shared memory (coalesced loads, the
// powers formed in the order of k_rfft_weight), then warp w transforms
// spectrum a0 + w.
constexpr int kWeightsMax = kMaxWeightDeg + 1;

__global__ void __launch_bounds__(256, 2)
k_rfft_weight_w(const uint8_t* __restrict__ Mfit, const float* __restrict__ S, const double* __restrict__ sky,
                const float* __restrict__ E, int H, int W, int a0, int na, float2* __restrict__ out,
                int64_t slab_stride, int64_t ccd_stride_out, const float2* __restrict__ twM,
                const float2* __restrict__ twN) {
  constexpr int M = 1024, NF = 2048, SROW = 33;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* g = reinterpret_cast<float*>(smem_raw);                                          // [na][NF]
  float2* tile = reinterpret_cast<float2*>(g + kWeightsMax * NF) + (threadIdx.x >> 5) * 32 * SROW;   // per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, ccd = blockIdx.z;
  TwReg tw;
  tw.load(twM, twN);
  const float sS = S ? (float)sky[2 * ccd + 1] : 0.f;
  const float xs = 2.f / (float)(W > 1 ? W - 1 : 1);
  for (int yy = 0; yy < kWarpRowsPerCta; ++yy) {
    const int y = blockIdx.x * kWarpRowsPerCta + yy;
    if (y >= H) break;   // uniform
    __syncthreads();     // the previous row's samples are transformed
    const int64_t roff = (int64_t)ccd * H * W + (int64_t)y * W;
    for (int x = threadIdx.x; x < NF; x += blockDim.x) {
      float fv = 0.f;
      if (x < W && Mfit[roff + x]) fv = S ? S[roff + x] - sS : (E ? E[roff + x] : 1.f);
      const float xt = (float)x * xs - 1.f;
      float pw = 1.f;   // xt^(a0 + i) as repeated products from 1, then times f
      for (int i = 0; i < a0; ++i) pw *= xt;
      for (int i = 0; i < na; ++i) {
        g[i * NF + x] = pw * fv;
        pw *= xt;
      }
    }
    __syncthreads();
    if (warp < na) {
      const float* gw = g + warp * NF;
      float2 v[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = *reinterpret_cast<const float2*>(gw + 2 * (lane + 32 * q));
      float2* o = out + (int64_t)ccd * ccd_stride_out + (int64_t)warp * slab_stride + (int64_t)y * M;
      warp_rfft2048_finish<false>(v, tile, tw, o, H);
    }
  }
}

template <typename T, int M>
static cudaError_t run_prod(const sfft_plan_s* p, const T* Rm, int d0, int nd, int self, c_t<T>* out,
                            int64_t slab_stride, int64_t ccd_stride) {
  using F = RowFFT<T, M>;
  auto kern = k_rfft_prod<T, M>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::smem_bytes());
  const int H = p->d.H;
  dim3 grid((H + F::RPB - 1) / F::RPB, self ? 1 : nd, p->d.batch);
  kern<<<grid, kFftThreads, F::smem_bytes(), p->stream>>>(Rm, H, p->d.W, p->d_dlist, d0, self, out, slab_stride,
                                                         ccd_stride, (const c_t<T>*)p->twM, (const c_t<T>*)p->twN);
  p->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T, int M>
static cudaError_t run_weight(const sfft_plan_s* p, const uint8_t* Mfit, const float* S, const double* sky,
                              const T* E, int a0, int na, c_t<T>* out, int64_t slab_stride, int64_t ccd_stride) {
  using F = RowFFT<T, M>;
  auto kern = k_rfft_weight<T, M>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::smem_bytes());
  const int H = p->d.H;
  dim3 grid((H + F::RPB - 1) / F::RPB, na, p->d.batch);
  kern<<<grid, kFftThreads, F::smem_bytes(), p->stream>>>(Mfit, S, sky, E, H, p->d.W, a0, out, slab_stride,
                                                         ccd_stride, (const c_t<T>*)p->twM, (const c_t<T>*)p->twN);
  p->nlaunch += 1;
  return cudaGetLastError();
}

#define SFFT_DISPATCH_M(MV, CALL)                    \
  switch (MV) {                                      \
    case 32: { constexpr int M = 32; return CALL; }  \
    case 64: { constexpr int M = 64; return CALL; }  \
    case 128: { constexpr int M = 128; return CALL; } \
    case 256: { constexpr int M = 256; return CALL; } \
    case 512: { constexpr int M = 512; return CALL; } \
    case 1024: { constexpr int M = 1024; return CALL; } \
    default: return cudaErrorInvalidValue;           \
  }

template <typename T, int M>
static cudaError_t run_prod_dy(const sfft_plan_s* p, const T* Rm, int nc, int d0, int nd, c_t<T>* out,
                               int64_t slab_stride, int64_t ccd_stride) {
  using F = RowFFT<T, M>;
  const size_t smem = F::smem_bytes() + sizeof(T) * (size_t)(2 * (2 * M) + 32);
  // product spectra [d][y][k], or k-slot-blocked [d][k / 16][y][k % 16] for
  // the lane-per-difference contraction
  auto kern = p->dl ? k_rfft_prod_dy<T, M, true> : k_rfft_prod_dy<T, M, false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int L = p->d.L;
  auto dy_of = [L](int id) { return id < L ? 0 : 1 + (id - L) / (2 * L - 1); };
  const int ndy = dy_of(d0 + nd - 1) - dy_of(d0) + 1;
  dim3 grid(p->d.H, ndy, nc);
  kern<<<grid, kFftThreads, smem, p->stream>>>(Rm, p->d.H, p->d.W, L, d0, nd, out, slab_stride, ccd_stride,
                                               (const c_t<T>*)p->twM, (const c_t<T>*)p->twN);
  p->nlaunch += 1;
  return cudaGetLastError();
}

static cudaError_t run_prod_dy_w(const sfft_plan_s* p, const float* Rm, int nc, int d0, int nd, float2* out,
                                 int64_t slab_stride, int64_t ccd_stride) {
  constexpr int NF = 2048;
  const size_t smem = sizeof(float) * (size_t)(2 * NF + 32) + sizeof(float2) * 8 * 32 * 33;
  auto kern = p->dl ? k_rfft_prod_dy_w<true> : k_rfft_prod_dy_w<false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int L = p->d.L;
  auto dy_of = [L](int id) { return id < L ? 0 : 1 + (id - L) / (2 * L - 1); };
  const int ndy = dy_of(d0 + nd - 1) - dy_of(d0) + 1;
  dim3 grid((p->d.H + kWarpRowsPerCta - 1) / kWarpRowsPerCta, ndy, nc);
  kern<<<grid, 256, smem, p->stream>>>(Rm, p->d.H, p->d.W, L, d0, nd, out, slab_stride, ccd_stride,
                                       (const float2*)p->twM, (const float2*)p->twN);
  p->nlaunch += 1;
  return cudaGetLastError();
}

template <typename T>
static cudaError_t prod_T(const sfft_plan_s* p, int c0, int nc, int d0, int nd, void* ws) {
  // R_m of the group's CCDs in; their product spectra to the group-local slabs
  const int64_t HM = (int64_t)p->d.H * p->M;
  const T* Rm = ws_at<T>(ws, p->rm) + (int64_t)c0 * p->d.H * p->d.W;
  c_t<T>* out = ws_at<c_t<T>>(ws, p->phat);
  if constexpr (sizeof(T) == 4) {
    if (p->M == 1024)
      return run_prod_dy_w(p, (const float*)Rm, nc, d0, nd, (float2*)out, HM, HM * p->d_batch);
  }
  SFFT_DISPATCH_M(p->M, (run_prod_dy<T, M>(p, Rm, nc, d0, nd, out, HM, HM * p->d_batch)))
}

template <typename T>
static cudaError_t rm_T(const sfft_plan_s* p, void* ws) {
  const int64_t HM = (int64_t)p->d.H * p->M;
  const T* Rm = ws_at<T>(ws, p->rm);
  c_t<T>* out = ws_at<c_t<T>>(ws, p->rhat);
  SFFT_DISPATCH_M(p->M, (run_prod<T, M>(p, Rm, 0, 1, 1, out, HM, HM)))
}

template <typename T>
static cudaError_t weights_T(const sfft_plan_s* p, const float* S, const void* eimg, int a0, int na, void* out,
                             int nslab, void* ws) {
  // `out` is the base of a region holding `nslab` spectra per CCD; slabs a0 .. a0+na-1 are written
  const int64_t HM = (int64_t)p->d.H * p->M;
  const uint8_t* Mfit = ws_at<uint8_t>(ws, p->mfit);
  const double* sky = ws_at<double>(ws, p->sky);
  if constexpr (sizeof(T) == 4) {
    if (p->M == 1024 && na <= kWeightsMax) {   // 2048-sample rows: the warp-per-row transform
      const size_t smem = sizeof(float) * kWeightsMax * 2048 + sizeof(float2) * 8 * 32 * 33;
      cudaFuncSetAttribute(k_rfft_weight_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      dim3 grid((p->d.H + kWarpRowsPerCta - 1) / kWarpRowsPerCta, 1, p->d.batch);
      k_rfft_weight_w<<<grid, 256, smem, p->stream>>>(Mfit, S, sky, (const float*)eimg, p->d.H, p->d.W, a0, na,
                                                     (float2*)out + a0 * HM, HM, HM * nslab, (const float2*)p->twM,
                                                     (const float2*)p->twN);
      p->nlaunch += 1;
      return cudaGetLastError();
    }
  }
  SFFT_DISPATCH_M(p->M, (run_weight<T, M>(p, Mfit, S, sky, (const T*)eimg, a0, na, (c_t<T>*)out + a0 * HM, HM,
                                          HM * nslab)))
}

cudaError_t launch_rfft_prod(const sfft_plan_s* p, int c0, int nc, int d0, int nd, void* ws) {
  return p->fp64 ? prod_T<double>(p, c0, nc, d0, nd, ws) : prod_T<float>(p, c0, nc, d0, nd, ws);
}
cudaError_t launch_rfft_rm(const sfft_plan_s* p, void* ws) {
  return p->fp64 ? rm_T<double>(p, ws) : rm_T<float>(p, ws);
}
cudaError_t launch_rfft_weights(const sfft_plan_s* p, const float* S, const void* eimg, int a0, int na, void* out,
                                int nslab, void* ws) {
  return p->fp64 ? weights_T<double>(p, S, eimg, a0, na, out, nslab, ws)
                 : weights_T<float>(p, S, eimg, a0, na, out, nslab, ws);
}

}  // namespace sfft
