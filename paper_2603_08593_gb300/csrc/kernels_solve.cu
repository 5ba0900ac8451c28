// Normal-matrix scatter and the FP64 solve.
//
// Scatter: A[(j,p),(j',p')] = g_{u_j - u_j', phi_p phi_p'}(u_j) for the kernel
// block (the half-plane entry or, for the other half plane, its mirror at lag
// u_j'), A[(j,p), q] = g^{KB}_{phi_p psi_q}(u_j), A[q, q'] = moment of
// M_fit psi_q psi_q', b_(j,p) = g^{bK}_p(u_j), b_q = moment of M_fit psi_q S'.
//
// Solve: Jacobi equilibration D_s = diag(A)^-1/2, right-looking blocked
// Cholesky (32 x 32 blocks: one launch factors the diagonal block and solves
// the panel below it, one launch applies the trailing update) of D_s A D_s,
// blocked forward and backward substitution, theta = D_s y.
// Per-CCD status flags (never a trap): 1 = not positive definite, 2 = non-finite.
#include "common.cuh"
#include "plan.h"

namespace sfft {

constexpr int NBK = 32;  // Cholesky block size

__device__ __forceinline__ void mono_expo(int p, int& a, int& b) {
  int n = 0;
  while ((n + 1) * (n + 2) / 2 <= p) ++n;
  b = p - n * (n + 1) / 2;
  a = n - b;
}

struct ScatterArgs {
  int L, w, NK, NB, NKK, N;
  int nm_kk, nm_kb, nm_bk, nm_bb;
  int64_t s_gkk, s_gkb, s_gbk, s_mbb, s_mb;   // per-CCD strides (doubles)
};

__global__ void __launch_bounds__(256)
k_scatter(ScatterArgs a, const double* __restrict__ gkk, const double* __restrict__ gkb,
          const double* __restrict__ gbk, const double* __restrict__ mbb, const double* __restrict__ mb,
          const int* __restrict__ hdidx, double* __restrict__ A, double* __restrict__ b, int rhs_only) {
  const int ccd = blockIdx.y;
  const int64_t NN = (int64_t)a.N * a.N;
  const int L = a.L, w = a.w, NK = a.NK;
  const double* Gkk = gkk + ccd * a.s_gkk;
  const double* Gkb = gkb + ccd * a.s_gkb;
  const double* Gbk = gbk + ccd * a.s_gbk;
  const double* Mbb = mbb + ccd * a.s_mbb;
  const double* Mb = mb + ccd * a.s_mb;
  const int64_t total = rhs_only ? a.N : NN + a.N;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    if (rhs_only || t >= NN) {
      const int r = (int)(rhs_only ? t : t - NN);
      double v;
      if (r < a.NKK) {
        const int j = r / NK, p = r % NK;
        v = Gbk[((j / L) * L + (j % L)) * a.nm_bk + p];
      } else {
        v = Mb[r - a.NKK];
      }
      b[(int64_t)ccd * a.N + r] = v;
      continue;
    }
    const int r = (int)(t / a.N), c = (int)(t % a.N);
    double v;
    if (r < a.NKK && c < a.NKK) {
      const int j = r / NK, p = r % NK, j2 = c / NK, p2 = c % NK;
      const int uy = j / L - w, ux = j % L - w, uy2 = j2 / L - w, ux2 = j2 % L - w;
      const int dy = uy - uy2, dx = ux - ux2;
      int ap, bp, aq, bq;
      mono_expo(p, ap, bp);
      mono_expo(p2, aq, bq);
      const int m = mono_index(ap + aq, bp + bq);
      int id = hdidx[(dy + L - 1) * (2 * L - 1) + (dx + L - 1)];
      if (id >= 0) {
        v = Gkk[(((int64_t)id * L + (uy + w)) * L + (ux + w)) * a.nm_kk + m];
      } else {
        id = hdidx[(-dy + L - 1) * (2 * L - 1) + (-dx + L - 1)];
        v = Gkk[(((int64_t)id * L + (uy2 + w)) * L + (ux2 + w)) * a.nm_kk + m];
      }
    } else if (r < a.NKK || c < a.NKK) {
      const int rk = r < a.NKK ? r : c, rb = r < a.NKK ? c : r;
      const int j = rk / NK, p = rk % NK, q = rb - a.NKK;
      int ap, bp, aq, bq;
      mono_expo(p, ap, bp);
      mono_expo(q, aq, bq);
      v = Gkb[j * a.nm_kb + mono_index(ap + aq, bp + bq)];
    } else {
      int ap, bp, aq, bq;
      mono_expo(r - a.NKK, ap, bp);
      mono_expo(c - a.NKK, aq, bq);
      v = Mbb[mono_index(ap + aq, bp + bq)];
    }
    A[(int64_t)ccd * NN + t] = v;
  }
}

// scale = diag(A)^-1/2; Lf (lower) = D_s A D_s; status flags
__global__ void __launch_bounds__(256)
k_chol_init(const double* __restrict__ A, double* __restrict__ Lf, double* __restrict__ scale,
            int* __restrict__ status, int N) {
  const int ccd = blockIdx.y;
  const int64_t NN = (int64_t)N * N;
  const double* a = A + ccd * NN;
  double* l = Lf + ccd * NN;
  double* s = scale + (int64_t)ccd * N;
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const double d = a[(int64_t)i * N + i];
      if (!isfinite(d)) atomicOr(&status[ccd], 2);
      else if (!(d > 0.0)) atomicOr(&status[ccd], 1);
    }
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < NN; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / N), j = (int)(t % N);
    if (j > i) continue;
    const double di = a[(int64_t)i * N + i], dj = a[(int64_t)j * N + j];
    const double si = di > 0.0 ? rsqrt(di) : 0.0, sj = dj > 0.0 ? rsqrt(dj) : 0.0;
    const double v = a[t];
    if (!isfinite(v)) atomicOr(&status[ccd], 2);
    l[t] = v * si * sj;
    if (i == j) s[i] = si;
  }
}

// Factor the diagonal block [kb, kb+nb) in shared memory (one warp, lane i
// owns row i) and solve this CTA's 32 panel rows r >= kb + nb against it:
// X = A_rk L_kk^-T.  Every panel CTA factors the small block itself, so one
// launch per block column does both; CTA 0 writes the factor back and reports
// a non-positive or non-finite pivot.  blockDim = 32.
__global__ void __launch_bounds__(NBK)
k_chol_panel(double* __restrict__ Lf, int* __restrict__ status, int N, int kb) {
  __shared__ double blk[NBK][NBK + 1];
  __shared__ double rdiag[NBK];   // 1 / L_cc
  const int ccd = blockIdx.y, lane = threadIdx.x;
  double* l = Lf + (int64_t)ccd * N * N;
  const int nb = min(NBK, N - kb);
  for (int i = 0; i < NBK; ++i) blk[i][lane] = (i < nb && lane <= i) ? l[(int64_t)(kb + i) * N + kb + lane] : 0.0;
  __syncwarp();
  bool bad = false, nonfinite = false;
  for (int c = 0; c < nb; ++c) {
    if (lane == c) {
      double d = blk[c][c];
      if (!(d > 0.0) || !isfinite(d)) { bad = true; nonfinite = !isfinite(d); d = 1.0; }
      const double s = sqrt(d);
      blk[c][c] = s;
      rdiag[c] = 1.0 / s;
    }
    __syncwarp();
    if (lane > c && lane < nb) blk[lane][c] *= rdiag[c];
    __syncwarp();
    if (lane > c && lane < nb) {
      const double lic = blk[lane][c];
      for (int j = c + 1; j <= lane; ++j) blk[lane][j] -= lic * blk[j][c];
    }
    __syncwarp();
  }
  if (blockIdx.x == 0) {
    if (bad) atomicOr(&status[ccd], nonfinite ? 2 : 1);
    for (int i = 0; i < nb; ++i)
      if (lane <= i) l[(int64_t)(kb + i) * N + kb + lane] = blk[i][lane];
  }
  const int r = kb + nb + blockIdx.x * NBK + lane;
  if (r >= N) return;
  double x[NBK];
  double* row = l + (int64_t)r * N + kb;
#pragma unroll
  for (int c = 0; c < NBK; ++c) x[c] = c < nb ? row[c] : 0.0;
#pragma unroll
  for (int c = 0; c < NBK; ++c) {
    if (c < nb) {
      // four independent partial sums keep the FP64 dependency chains short
      double v0 = x[c], v1 = 0.0, v2 = 0.0, v3 = 0.0;
#pragma unroll
      for (int t = 0; t + 3 < c; t += 4) {
        v0 -= x[t] * blk[c][t];
        v1 -= x[t + 1] * blk[c][t + 1];
        v2 -= x[t + 2] * blk[c][t + 2];
        v3 -= x[t + 3] * blk[c][t + 3];
      }
#pragma unroll
      for (int t = c & ~3; t < c; ++t) v0 -= x[t] * blk[c][t];
      x[c] = ((v0 + v1) + (v2 + v3)) * rdiag[c];
    }
  }
#pragma unroll
  for (int c = 0; c < NBK; ++c) if (c < nb) row[c] = x[c];
}

// trailing update of lower tiles (bi >= bj) below the panel: C -= P_i P_j^T
__global__ void __launch_bounds__(256)
k_chol_update(double* __restrict__ Lf, int N, int kb) {
  __shared__ double Pi[NBK][NBK + 1], Pj[NBK][NBK + 1];
  const int ccd = blockIdx.y;
  double* l = Lf + (int64_t)ccd * N * N;
  const int nb = min(NBK, N - kb);
  const int r0 = kb + nb;
  // linear tile index -> (bi, bj), bj <= bi
  int t = blockIdx.x, bi = 0;
  while (t > bi) { t -= bi + 1; ++bi; }
  const int bj = t;
  const int i0 = r0 + bi * NBK, j0 = r0 + bj * NBK;
  for (int q = threadIdx.x; q < NBK * NBK; q += blockDim.x) {
    const int i = q / NBK, c = q % NBK;
    Pi[i][c] = (i0 + i < N && c < nb) ? l[(int64_t)(i0 + i) * N + kb + c] : 0.0;
    Pj[i][c] = (j0 + i < N && c < nb) ? l[(int64_t)(j0 + i) * N + kb + c] : 0.0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NBK * NBK; q += blockDim.x) {
    const int i = q / NBK, j = q % NBK;
    const int gi = i0 + i, gj = j0 + j;
    if (gi >= N || gj >= N || gj > gi) continue;
    double s = 0.0;
#pragma unroll 8
    for (int c = 0; c < NBK; ++c) s += Pi[i][c] * Pj[j][c];
    l[(int64_t)gi * N + gj] -= s;
  }
}

// x = D_s (L L^T)^-1 D_s rhs, one CTA per CCD.  Blocked substitution: each
// 32 x 32 diagonal block is solved by one warp from shared memory (lane i owns
// unknown i, one shuffle per column), the coupling to the remaining unknowns
// is applied by all threads, one unknown per thread.
__global__ void __launch_bounds__(1024)
k_chol_solve(const double* __restrict__ Lf, const double* __restrict__ scale, const double* __restrict__ rhs,
             double* __restrict__ x, int N, int* __restrict__ status) {
  extern __shared__ double sh[];   // y[N]
  __shared__ double ld[32][33];
  const int ccd = blockIdx.x;
  const double* l = Lf + (int64_t)ccd * N * N;
  const double* s = scale + (int64_t)ccd * N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < N; i += blockDim.x) sh[i] = rhs[(int64_t)ccd * N + i] * s[i];
  const int nblk = (N + 31) / 32;
  // forward: L y = r
  for (int bi = 0; bi < nblk; ++bi) {
    const int jb = bi * 32, nb = min(32, N - jb);
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
      const int i = t >> 5, j = t & 31;
      ld[i][j] = (i < nb && j <= i) ? l[(int64_t)(jb + i) * N + jb + j] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double y = lane < nb ? sh[jb + lane] : 0.0;
      const double rd = lane < nb ? 1.0 / ld[lane][lane] : 0.0;
      for (int c = 0; c < nb; ++c) {
        if (lane == c) y *= rd;
        const double yc = __shfl_sync(0xffffffffu, y, c);
        if (lane > c) y -= ld[lane][c] * yc;
      }
      if (lane < nb) sh[jb + lane] = y;
    }
    __syncthreads();
    for (int i = jb + nb + threadIdx.x; i < N; i += blockDim.x) {
      const double* row = l + (int64_t)i * N + jb;
      double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
      int c = 0;
      for (; c + 3 < nb; c += 4) {
        v0 += row[c] * sh[jb + c];
        v1 += row[c + 1] * sh[jb + c + 1];
        v2 += row[c + 2] * sh[jb + c + 2];
        v3 += row[c + 3] * sh[jb + c + 3];
      }
      for (; c < nb; ++c) v0 += row[c] * sh[jb + c];
      sh[i] -= (v0 + v1) + (v2 + v3);
    }
    __syncthreads();
  }
  // backward: L^T z = y
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int jb = bi * 32, nb = min(32, N - jb);
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
      const int i = t >> 5, j = t & 31;
      ld[i][j] = (i < nb && j <= i) ? l[(int64_t)(jb + i) * N + jb + j] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double z = lane < nb ? sh[jb + lane] : 0.0;
      const double rd = lane < nb ? 1.0 / ld[lane][lane] : 0.0;
      for (int c = nb - 1; c >= 0; --c) {
        if (lane == c) z *= rd;
        const double zc = __shfl_sync(0xffffffffu, z, c);
        if (lane < c) z -= ld[c][lane] * zc;
      }
      if (lane < nb) sh[jb + lane] = z;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < jb; i += blockDim.x) {
      double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
      int c = 0;
      for (; c + 3 < nb; c += 4) {
        v0 += l[(int64_t)(jb + c) * N + i] * sh[jb + c];
        v1 += l[(int64_t)(jb + c + 1) * N + i] * sh[jb + c + 1];
        v2 += l[(int64_t)(jb + c + 2) * N + i] * sh[jb + c + 2];
        v3 += l[(int64_t)(jb + c + 3) * N + i] * sh[jb + c + 3];
      }
      for (; c < nb; ++c) v0 += l[(int64_t)(jb + c) * N + i] * sh[jb + c];
      sh[i] -= (v0 + v1) + (v2 + v3);
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double v = sh[i] * s[i];
    if (!isfinite(v)) atomicOr(&status[ccd], 2);
    x[(int64_t)ccd * N + i] = v;
  }
}

__global__ void k_theta_finish(const double* __restrict__ x, double* __restrict__ theta_off, int N, int batch, int add) {
  const int64_t n = (int64_t)N * batch;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    theta_off[t] = add ? theta_off[t] + x[t] : x[t];
}

// background between offset and original units: B = B' + s_S - s_R sum_j K_j (q < N_K share phi_q)
__global__ void k_theta_units(const double* __restrict__ src, double* __restrict__ dst, const double* __restrict__ sky,
                              int L, int NK, int NB, int to_orig) {
  const int ccd = blockIdx.x;
  const int N = L * L * NK + NB, NKK = L * L * NK;
  const double* s = src + (int64_t)ccd * N;
  double* d = dst + (int64_t)ccd * N;
  const double sR = sky[2 * ccd], sS = sky[2 * ccd + 1];
  const double sg = to_orig ? 1.0 : -1.0;
  for (int i = threadIdx.x; i < NKK; i += blockDim.x) d[i] = s[i];
  for (int q = threadIdx.x; q < NB; q += blockDim.x) {
    double v = s[NKK + q];
    if (q == 0) v += sg * sS;
    if (q < NK) {
      double ks = 0.0;
      for (int j = 0; j < L * L; ++j) ks += s[j * NK + q];
      v -= sg * sR * ks;
    }
    d[NKK + q] = v;
  }
}

__global__ void k_info(const int* __restrict__ status, int32_t* __restrict__ info, int batch) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= batch) return;
  const int s = status[c];
  info[c] = (s & 2) ? SFFT_ERR_NONFINITE : ((s & 1) ? SFFT_ERR_SINGULAR : (s & 4 ? SFFT_ERR_TIMEOUT : SFFT_OK));
}

__global__ void k_kernel_at(const double* __restrict__ theta, double* __restrict__ K, int L, int DK, int NK, int NB,
                            double xt, double yt) {
  const int ccd = blockIdx.x;
  const int N = L * L * NK + NB;
  for (int j = threadIdx.x; j < L * L; j += blockDim.x) {
    double v = 0.0;
    for (int p = 0; p < NK; ++p) {
      int a, b;
      mono_expo(p, a, b);
      double f = 1.0;
      for (int i = 0; i < a; ++i) f *= xt;
      for (int i = 0; i < b; ++i) f *= yt;
      v += theta[(int64_t)ccd * N + j * NK + p] * f;
    }
    K[(int64_t)ccd * L * L + j] = v;
  }
}

// ------------------------------------------------------------------ launchers
cudaError_t launch_scatter(const sfft_plan_s* p, double* A, double* b, void* ws, bool rhs_only, double* rhs_out) {
  ScatterArgs a;
  a.L = p->d.L; a.w = p->w; a.NK = p->NK; a.NB = p->NB; a.NKK = p->NKK; a.N = p->N;
  a.nm_kk = n_mono(p->DM_KK); a.nm_kb = n_mono(p->DM_KB); a.nm_bk = n_mono(p->DM_bK); a.nm_bb = n_mono(p->DM_BB);
  const int LL = p->d.L * p->d.L;
  a.s_gkk = (int64_t)p->n_hd * LL * a.nm_kk;
  a.s_gkb = (int64_t)LL * a.nm_kb;
  a.s_gbk = (int64_t)LL * a.nm_bk;
  a.s_mbb = a.nm_bb;
  a.s_mb = n_mono(p->d.DB);
  const int64_t total = rhs_only ? p->N : (int64_t)p->N * p->N + p->N;
  int gx = (int)((total + 255) / 256);
  if (gx > 2048) gx = 2048;
  dim3 grid(gx, p->d.batch);
  k_scatter<<<grid, 256, 0, p->stream>>>(a, ws_at<double>(ws, p->gkk), ws_at<double>(ws, p->gkb),
                                         ws_at<double>(ws, p->gbk), ws_at<double>(ws, p->mom_bb),
                                         ws_at<double>(ws, p->mom_b), p->d_hdidx, A, rhs_only ? rhs_out : b,
                                         rhs_only ? 1 : 0);
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_cholesky(const sfft_plan_s* p, const double* A, void* ws) {
  const int N = p->N, B = p->d.batch;
  double* Lf = ws_at<double>(ws, p->lfac);
  double* scale = ws_at<double>(ws, p->scale);
  int* status = ws_at<int>(ws, p->status);
  dim3 gi(64, B);
  k_chol_init<<<gi, 256, 0, p->stream>>>(A, Lf, scale, status, N);
  p->nlaunch += 1;
  for (int kb = 0; kb < N; kb += NBK) {
    const int nb = N - kb < NBK ? N - kb : NBK;
    const int rem = N - kb - nb;
    const int T = (rem + NBK - 1) / NBK;
    k_chol_panel<<<dim3(T > 0 ? T : 1, B), NBK, 0, p->stream>>>(Lf, status, N, kb);
    p->nlaunch += 1;
    if (rem > 0) {
      k_chol_update<<<dim3(T * (T + 1) / 2, B), 256, 0, p->stream>>>(Lf, N, kb);
      p->nlaunch += 1;
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_chol_solve(const sfft_plan_s* p, const double* rhs, double* x, void* ws) {
  const int N = p->N;
  const size_t smem = sizeof(double) * N;
  cudaFuncSetAttribute(k_chol_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_chol_solve<<<p->d.batch, 1024, smem, p->stream>>>(ws_at<double>(ws, p->lfac), ws_at<double>(ws, p->scale), rhs,
                                                      x, N, ws_at<int>(ws, p->status));
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_theta_finish(const sfft_plan_s* p, const double* x, double* theta_off, bool add) {
  const int64_t n = (int64_t)p->N * p->d.batch;
  k_theta_finish<<<(int)((n + 255) / 256), 256, 0, p->stream>>>(x, theta_off, p->N, p->d.batch, add ? 1 : 0);
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_theta_to_orig(const sfft_plan_s* p, const double* theta_off, double* theta, void* ws) {
  k_theta_units<<<p->d.batch, 128, 0, p->stream>>>(theta_off, theta, ws_at<double>(ws, p->sky), p->d.L, p->NK, p->NB, 1);
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_theta_to_off(const sfft_plan_s* p, const double* theta, const double* sky, double* theta_off,
                                void* ws) {
  k_theta_units<<<p->d.batch, 128, 0, p->stream>>>(theta, theta_off, sky ? sky : ws_at<double>(ws, p->sky), p->d.L,
                                                   p->NK, p->NB, 0);
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_theta_units_raw(cudaStream_t s, const double* src, double* dst, const double* sky, int L, int NK,
                                   int NB, int batch, int to_orig) {
  k_theta_units<<<batch, 128, 0, s>>>(src, dst, sky, L, NK, NB, to_orig);
  return cudaGetLastError();
}

cudaError_t launch_info(const sfft_plan_s* p, int32_t* info, void* ws) {
  k_info<<<(p->d.batch + 127) / 128, 128, 0, p->stream>>>(ws_at<int>(ws, p->status), info, p->d.batch);
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_kernel_at(const sfft_plan_s* p, const double* theta, double x, double y, double* K) {
  const double xt = 2.0 * x / (double)(p->d.W > 1 ? p->d.W - 1 : 1) - 1.0;
  const double yt = 2.0 * y / (double)(p->d.H > 1 ? p->d.H - 1 : 1) - 1.0;
  k_kernel_at<<<p->d.batch, 128, 0, p->stream>>>(theta, K, p->d.L, p->d.DK, p->NK, p->NB, xt, yt);
  p->nlaunch += 1;
  return cudaGetLastError();
}

}  // namespace sfft
