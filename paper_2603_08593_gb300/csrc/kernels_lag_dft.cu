// Lags u_x of the lane-per-difference contraction's k-slot products
// (kernels_contract_dlane.cu), into the FP64 G arrays of the KK block.
#include "common.cuh"
#include "plan.h"

namespace sfft {

// Lags u_x of the k-slot products: for pair (d, u_y) of the difference batch,
// G[d][u_y][u_x][m] += (1/N_f) sum_{k=1}^{M-1} (C_Re 2 cos(2 pi k u_x / N_f)
// + C_Im 2 sin(2 pi k u_x / N_f)); slot 0 (the packed real bins) is summed by
// k_contract_slot0.  Lane (g, q) of warp v takes monomials 4q .. 4q + 3 (one
// float4 of the k-row's real parts and one of its imaginary parts) and the
// k-slots k = 1 + 8v + g (mod 64).  For |u_x| = 1 .. 5 it keeps the pair
// (sum C_Re cos, sum C_Im sin), one packed FMA per (k, monomial, |u_x|), whose
// sum and difference are the lags +|u_x| and -|u_x| (cos is even in u_x, sin
// odd).  The twiddles of a k are loaded once for its four monomials.  Sums
// are FP32 within a warp (16 k-slots per lane, then a tree over the warp's 8
// k-groups) and FP64 across the 8 warps: GB300's FP64 pipe retires about two
// operations per SM per clock, so FP64 stays out of the per-slot work.
template <int DM>
__global__ void __launch_bounds__(256, 2)
k_lag_dft(const int4* __restrict__ pairs, const char* __restrict__ cbuf0, size_t cbuf_ccd, double* __restrict__ g0,
          size_t g_ccd, int M, int Nf, int L, int dstride, const float2* __restrict__ twD) {
  // blockIdx.y: the CCD within its group (k-slot products); g0 points at the group's first CCD
  constexpr int NMONO = n_mono(DM);
  constexpr int NV = (kMaxL + 1) / 2;   // |u_x| = 0 .. 5
  constexpr int KG = 64, RUN = 4;
  __shared__ float red[8][16][kMaxL];
  const int4 pq = pairs[blockIdx.x];
  const int ccd = blockIdx.y, w = (L - 1) / 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = lane & 3, kg = warp * 8 + (lane >> 2);
  const float* C = reinterpret_cast<const float*>(cbuf0 + (size_t)ccd * cbuf_ccd) +
                   ((int64_t)pq.x * L + (pq.y + w)) * 32 + 4 * q;
  const int64_t kstride = (int64_t)dstride * L * 32;
  float s0[4];         // sum C_Re (u_x = 0)
  float2 sv[4][NV];    // [monomial][|u_x|]: (sum C_Re cos, sum C_Im sin); index 0 unused
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    s0[i] = 0.f;
#pragma unroll
    for (int v = 0; v < NV; ++v) sv[i][v] = make_float2(0.f, 0.f);
  }
  for (int kb = 1 + kg; kb < M; kb += KG * RUN) {
    float4 re[RUN], im[RUN];
#pragma unroll
    for (int t = 0; t < RUN; ++t) {
      const int k = kb + KG * t;
      const float4* ck = reinterpret_cast<const float4*>(C + (int64_t)(k < M ? k : 0) * kstride);
      re[t] = k < M ? __ldg(ck) : make_float4(0.f, 0.f, 0.f, 0.f);
      im[t] = k < M ? __ldg(ck + 4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int t = 0; t < RUN; ++t) {
      const int k = kb + KG * t;   // past the row: zero products, any twiddle
      float2 tw[NV];
#pragma unroll
      for (int v = 1; v < NV; ++v) tw[v] = __ldg(twD + ((k * v) & (Nf - 1)));
      const float cr[4] = {re[t].x, re[t].y, re[t].z, re[t].w};
      const float ci[4] = {im[t].x, im[t].y, im[t].z, im[t].w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        s0[i] += cr[i];
        const float2 c = make_float2(cr[i], ci[i]);
#pragma unroll
        for (int v = 1; v < NV; ++v) sv[i][v] = __ffma2_rn(c, tw[v], sv[i][v]);
      }
    }
  }
  // the warp's 8 k-groups (lanes with the same q)
#pragma unroll
  for (int o = 4; o < 32; o <<= 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      s0[i] += __shfl_xor_sync(0xffffffffu, s0[i], o);
#pragma unroll
      for (int v = 1; v < NV; ++v) {
        sv[i][v].x += __shfl_xor_sync(0xffffffffu, sv[i][v].x, o);
        sv[i][v].y += __shfl_xor_sync(0xffffffffu, sv[i][v].y, o);
      }
    }
  }
  if (lane < 4) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float* r = red[warp][4 * q + i];
      r[w] = s0[i];
#pragma unroll
      for (int v = 1; v < NV; ++v)
        if (v <= w) {
          r[w + v] = sv[i][v].x + sv[i][v].y;
          r[w - v] = sv[i][v].x - sv[i][v].y;
        }
    }
  }
  __syncthreads();
  // factor 2 of the one-sided sum and 1/N_f: a power of two, exact
  const double scale = 2.0 / (double)Nf;
  for (int t = threadIdx.x; t < 16 * L; t += blockDim.x) {
    const int mm = t % 16, xi = t / 16, ux = xi - w;
    if (mm >= NMONO || ux < pq.z || ux > pq.w) continue;
    double s = 0.0;
#pragma unroll
    for (int v = 0; v < 8; ++v) s += (double)red[v][mm][xi];
    g0[(size_t)ccd * g_ccd + (((int64_t)pq.x * L + (pq.y + w)) * L + xi) * NMONO + mm] += s * scale;
  }
}

template <int DM>
static cudaError_t lag_dft_dm(const sfft_plan_s* p, int batch_index, int c0, int nc, void* ws) {
  const int pair0 = p->dlp_first[batch_index], npair = p->dlp_count[batch_index];
  if (npair <= 0 || nc <= 0) return cudaSuccess;
  const int L = p->d.L;
  const size_t cbuf_ccd = (size_t)p->M * p->d_batch * L * 32 * sizeof(float);
  const size_t g_ccd = (size_t)p->n_hd * L * L * n_mono(DM);
  double* g0 = ws_at<double>(ws, p->gkk) + (size_t)c0 * g_ccd + (size_t)batch_index * p->d_batch * L * L * n_mono(DM);
  dim3 grid(npair, nc);
  k_lag_dft<DM><<<grid, 256, 0, p->stream>>>(p->d_dlpairs + pair0, static_cast<char*>(ws) + p->cbuf.off, cbuf_ccd,
                                             g0, g_ccd, p->M, p->Nf, L, p->d_batch, (const float2*)p->twD);
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_lag_dft(const sfft_plan_s* p, int batch_index, int c0, int nc, void* ws) {
  switch (p->DM_KK) {
    case 0: return lag_dft_dm<0>(p, batch_index, c0, nc, ws);
    case 2: return lag_dft_dm<2>(p, batch_index, c0, nc, ws);
    case 4: return lag_dft_dm<4>(p, batch_index, c0, nc, ws);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sfft
