// Lags u_x of the lane-per-difference contraction's k-slot products
// (kernels_contract_dlane.cu), into the FP64 G arrays of the KK block.
#include "common.cuh"
#include "plan.h"

namespace sfft {

// Lags u_x of the k-slot products: for pair (d, u_y) of the difference batch,
// G[d][u_y][u_x][m] += (1/N_f) sum_{k=1}^{M-1} (C_Re 2 cos(2 pi k u_x / N_f)
// + C_Im 2 sin(2 pi k u_x / N_f)); slot 0 (the packed real bins) is summed by
// k_contract_slot0.  Thread (m, g) takes the k-slots k = 1 + g (mod 16) for
// every u_x (cos is even and sin odd in u_x), in FP32 runs of 16 slots added
// to FP64; the 16 groups are then summed in FP64 in a fixed order.
template <int DM>
__global__ void __launch_bounds__(256)
k_lag_dft(const int4* __restrict__ pairs, const char* __restrict__ cbuf0, size_t cbuf_ccd, double* __restrict__ g0,
          size_t g_ccd, int M, int Nf, int L, int dstride, const float2* __restrict__ twD) {
  // blockIdx.y: the CCD within its group (k-slot products); g0 points at the group's first CCD
  constexpr int NMONO = n_mono(DM);
  constexpr int NG = 16, W5 = (kMaxL - 1) / 2;
  __shared__ double red[NG][16][kMaxL];
  const int4 pq = pairs[blockIdx.x];
  const int ccd = blockIdx.y, w = (L - 1) / 2;
  const int m = threadIdx.x & 15, grp = threadIdx.x >> 4;
  const float* C = reinterpret_cast<const float*>(cbuf0 + (size_t)ccd * cbuf_ccd) +
                   ((int64_t)pq.x * L + (pq.y + w)) * 32;
  const int64_t kstride = (int64_t)dstride * L * 32;
  double sp[W5 + 1], sn[W5 + 1];   // u_x = +v and -v
  float fp[W5 + 1], fn[W5 + 1];
#pragma unroll
  for (int v = 0; v <= W5; ++v) { sp[v] = sn[v] = 0.0; fp[v] = fn[v] = 0.f; }
  // runs of 16 k-slots per thread: the run's 32 loads are issued together,
  // then summed in FP32 and added to the FP64 totals
  constexpr int RUN = 16;
  for (int kb = 1 + grp; kb < M; kb += NG * RUN) {
    float cr[RUN], ci[RUN];
#pragma unroll
    for (int t = 0; t < RUN; ++t) {
      const int k = kb + NG * t;
      const float* ck = C + (int64_t)(k < M ? k : 0) * kstride;
      cr[t] = k < M ? __ldg(ck + m) : 0.f;
      ci[t] = k < M ? __ldg(ck + 16 + m) : 0.f;
    }
#pragma unroll
    for (int t = 0; t < RUN; ++t) {
      const int k = kb + NG * t;
#pragma unroll
      for (int v = 0; v <= W5; ++v) {
        if (v > w) break;
        const float2 tw = __ldg(twD + ((k * v) & (Nf - 1)));
        const float a = cr[t] * tw.x, b = ci[t] * tw.y;
        fp[v] += 2.f * (a + b);
        fn[v] += 2.f * (a - b);
      }
    }
#pragma unroll
    for (int v = 0; v <= W5; ++v) { sp[v] += fp[v]; sn[v] += fn[v]; fp[v] = fn[v] = 0.f; }
  }
#pragma unroll
  for (int v = 0; v <= W5; ++v) {
    sp[v] += fp[v];
    sn[v] += fn[v];
    if (v <= w) {
      red[grp][m][w + v] = sp[v];
      red[grp][m][w - v] = sn[v];   // u_x = 0 writes the same value twice
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 16 * L; t += blockDim.x) {
    const int mm = t % 16, xi = t / 16, ux = xi - w;
    if (mm >= NMONO || ux < pq.z || ux > pq.w) continue;
    double s = 0.0;
    for (int g = 0; g < NG; ++g) s += red[g][mm][xi];
    g0[(size_t)ccd * g_ccd + (((int64_t)pq.x * L + (pq.y + w)) * L + xi) * NMONO + mm] += s / (double)Nf;
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
