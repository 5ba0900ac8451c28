// Normal-matrix scatter and the FP64 solve.
//
// Scatter: A[(j,p),(j',p')] = g_{u_j - u_j', phi_p phi_p'}(u_j) for the kernel
// block (the half-plane entry or, for the other half plane, its mirror at lag
// u_j'), A[(j,p), q] = g^{KB}_{phi_p psi_q}(u_j), A[q, q'] = moment of
// M_fit psi_q psi_q', b_(j,p) = g^{bK}_p(u_j), b_q = moment of M_fit psi_q S'.
//
// Solve: optionally the constant-ratio projection T A T^T (below), then
// Jacobi equilibration D_s = diag(A)^-1/2, right-looking blocked
// Cholesky of D_s A D_s (32 x 32 blocks, all block steps in one cooperative
// launch), blocked forward and backward substitution with the inverted
// diagonal blocks, theta = D_s y.
// Per-CCD status flags (never a trap): 1 = not positive definite, 2 = non-finite.
#include <algorithm>

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

// ---------------------------------------------------------------- constant photometric ratio
// With the kernel sum held constant over the chip the solved unknowns are,
// in order, c[u, p] for the offsets u != 0 (j ascending, p minor), the
// constant a_0 of delta_0 and the N_B background terms, the basis
// K = a_0 delta_0 + sum_{u != 0} sum_p c[u, p] phi_p (delta_u - delta_0).
// The full-layout coefficients are theta = T^T theta_c, where T's row of
// c[u, p] is e_(u,p) - e_(0,p), its row of a_0 is e_(0,0) and the background
// rows are the identity, so the constrained normal equations are
// (T A T^T) theta_c = T b.  Each row of T has at most two non-zeros.
struct CprMap {
  int on;    // 0: the free fit (T = identity)
  int NK;    // kernel polynomial terms
  int jc;    // index of the zero offset, (L^2 - 1) / 2
  int nkc;   // (L^2 - 1) N_K
};

// Columns (full layout) and signs of row r of T; returns their count.
__device__ __forceinline__ int cpr_row(const CprMap& m, int r, int* idx, double* sg) {
  if (!m.on) { idx[0] = r; sg[0] = 1.0; return 1; }
  if (r < m.nkc) {
    const int jj = r / m.NK, p = r % m.NK;
    idx[0] = (jj < m.jc ? jj : jj + 1) * m.NK + p; sg[0] = 1.0;
    idx[1] = m.jc * m.NK + p; sg[1] = -1.0;
    return 2;
  }
  idx[0] = r == m.nkc ? m.jc * m.NK : r - 1 + m.NK;
  sg[0] = 1.0;
  return 1;
}

// (T A T^T)[i][j] from the full matrix a (row stride N)
__device__ __forceinline__ double cpr_entry(const double* a, int64_t N, const CprMap& m, int i, int j) {
  int ii[2], jj[2];
  double si[2], sj[2];
  const int ni = cpr_row(m, i, ii, si), nj = cpr_row(m, j, jj, sj);
  double v = 0.0;
  for (int x = 0; x < ni; ++x)
    for (int y = 0; y < nj; ++y) v += si[x] * sj[y] * a[(int64_t)ii[x] * N + jj[y]];
  return v;
}

// out = T b (per CCD: b stride N, out stride Ns)
__global__ void k_cpr_rhs(const double* __restrict__ b, double* __restrict__ out, int N, int Ns, CprMap m) {
  const int ccd = blockIdx.y;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < Ns; r += gridDim.x * blockDim.x) {
    int idx[2];
    double sg[2];
    const int n = cpr_row(m, r, idx, sg);
    double v = 0.0;
    for (int x = 0; x < n; ++x) v += sg[x] * b[(int64_t)ccd * N + idx[x]];
    out[(int64_t)ccd * Ns + r] = v;
  }
}

// theta_off (=|+=) T^T x (per CCD: x stride Ns, theta_off stride N)
__global__ void k_cpr_expand(const double* __restrict__ x, double* __restrict__ theta_off, int N, int Ns, CprMap m,
                             int add) {
  const int ccd = blockIdx.y;
  const double* xc = x + (int64_t)ccd * Ns;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double v;
    if (i >= m.nkc + m.NK) {
      v = xc[i - m.NK + 1];                      // background
    } else {
      const int j = i / m.NK, p = i % m.NK;
      if (j != m.jc) {
        v = xc[(j < m.jc ? j : j - 1) * m.NK + p];
      } else {
        v = p == 0 ? xc[m.nkc] : 0.0;
        for (int jj = 0; jj < m.nkc / m.NK; ++jj) v -= xc[jj * m.NK + p];
      }
    }
    double* o = theta_off + (int64_t)ccd * N + i;
    *o = add ? *o + v : v;
  }
}

// scale = diag(A_s)^-1/2; Lf (lower) = D_s A_s D_s; status flags.  A_s is the
// solved system: A itself (row stride N = Ns) or T A T^T (size Ns).
__global__ void __launch_bounds__(256)
k_chol_init(const double* __restrict__ A, double* __restrict__ Lf, double* __restrict__ scale,
            int* __restrict__ status, int N, int Ns, CprMap m) {
  const int ccd = blockIdx.y;
  const int64_t NS2 = (int64_t)Ns * Ns;
  const double* a = A + ccd * (int64_t)N * N;
  double* l = Lf + ccd * NS2;
  double* s = scale + (int64_t)ccd * Ns;
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < Ns; i += blockDim.x) {
      const double d = cpr_entry(a, N, m, i, i);
      if (!isfinite(d)) atomicOr(&status[ccd], 2);
      else if (!(d > 0.0)) atomicOr(&status[ccd], 1);
    }
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < NS2; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / Ns), j = (int)(t % Ns);
    if (j > i) continue;
    const double di = cpr_entry(a, N, m, i, i), dj = cpr_entry(a, N, m, j, j);
    const double si = di > 0.0 ? rsqrt(di) : 0.0, sj = dj > 0.0 ? rsqrt(dj) : 0.0;
    const double v = cpr_entry(a, N, m, i, j);
    if (!isfinite(v)) atomicOr(&status[ccd], 2);
    l[t] = v * si * sj;
    if (i == j) s[i] = si;
  }
}

// ---------------------------------------------------------------- persistent blocked Cholesky
// One cooperative launch factors every CCD's matrix.  For each 32-column
// block k: (A) one CTA per CCD factors the diagonal block in shared memory and
// inverts the factor; (B) all CTAs take 32-row tiles of the panels below the
// diagonal blocks and multiply them by the transposed inverse (the panel
// triangular solve as a product); (C) all CTAs take 32 x 32 tiles of the
// trailing lower triangles and subtract P_i P_j^T, and the CTA that updates
// the next diagonal block factors it at once (A of step k + 1, overlapped
// with the rest of C).  The phases are separated
// by a grid-wide barrier whose waits are bounded: a barrier that gives up (or
// sees another CTA give up) flags every CCD with bit 4 and the kernel returns.
// The inverses of the diagonal blocks are kept for the substitutions.  Data
// written by other CTAs is read with L2-coherent loads (ld.global.cg).
struct GridBar { unsigned count, gen, abort, pad; };

constexpr int kBarSpin = 1 << 24;   // x >= 64 ns per try: about a second

__device__ bool grid_sync_bounded(GridBar* bar, int* flag_sh) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &bar->gen;
    volatile unsigned* vab = &bar->abort;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u) + 1u;
    bool ok = true;
    if (arrived == gridDim.x) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      for (int it = 0; *vgen == g; ++it) {
        if (*vab != 0u || it > kBarSpin) { ok = false; break; }
        __nanosleep(64);
      }
    }
    if (!ok) atomicExch(&bar->abort, 1u);
    __threadfence();
    *flag_sh = ok ? 1 : 0;
  }
  __syncthreads();
  return *flag_sh != 0;
}

// Factor the diagonal block [kb, kb + nb) of one CCD with the whole CTA
// (identity-padded past nb), write the factor back and its inverse (32 x 32,
// lower) to `inv_out`.  Pivots use the reciprocal square root, so neither a
// square root nor a division sits on the column-to-column dependency chain.
// A non-positive or non-finite pivot is replaced by 1 and reported in the
// CCD's status word.
__device__ void factor_diag(double* __restrict__ l, double* __restrict__ inv_out, int* __restrict__ st, int N, int kb,
                            int nb, double (*blk)[NBK + 1], double (*inv)[NBK + 1], double* rinv) {
  const int tid = threadIdx.x;
  for (int e = tid; e < NBK * NBK; e += blockDim.x) {
    const int i = e / NBK, j = e % NBK;
    blk[i][j] = (i < nb && j <= i) ? __ldcg(l + (int64_t)(kb + i) * N + kb + j) : (i == j ? 1.0 : 0.0);
    inv[i][j] = i == j ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < NBK; ++c) {
    if (tid == 0) {
      double d = blk[c][c];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicOr(st, isfinite(d) ? 1 : 2);
        d = 1.0;
      }
      const double r = rsqrt(d);
      blk[c][c] = d * r;
      rinv[c] = r;
    }
    __syncthreads();
    if (tid > c && tid < NBK) blk[tid][c] *= rinv[c];
    __syncthreads();
    for (int e = tid; e < NBK * NBK; e += blockDim.x) {
      const int i = e / NBK, j = e % NBK;
      if (j > c && j <= i) blk[i][j] -= blk[i][c] * blk[j][c];
    }
    __syncthreads();
  }
  // L X = I by row elimination: row t is final once scaled, then removed below
  for (int t = 0; t < NBK; ++t) {
    if (tid <= t) inv[t][tid] *= rinv[t];
    __syncthreads();
    for (int e = tid; e < NBK * NBK; e += blockDim.x) {
      const int i = e / NBK, j = e % NBK;
      if (i > t && j <= t) inv[i][j] -= blk[i][t] * inv[t][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < NBK * NBK; e += blockDim.x) {
    const int i = e / NBK, j = e % NBK;
    inv_out[e] = inv[i][j];
    if (i < nb && j <= i) l[(int64_t)(kb + i) * N + kb + j] = blk[i][j];
  }
}

__global__ void __launch_bounds__(256)
k_chol_coop(double* __restrict__ Lf, double* __restrict__ dinv, int* __restrict__ status, int N, int B,
            GridBar* __restrict__ bar) {
  __shared__ double sa[NBK][NBK + 1], sb[NBK][NBK + 1];
  __shared__ double rinv[NBK];
  __shared__ int flag;
  const int nblk = (N + NBK - 1) / NBK;
  const int64_t NN = (int64_t)N * N;
  const int tid = threadIdx.x;
  // (A) of block 0; later diagonal blocks are factored as soon as their last
  // trailing update lands (look-ahead inside phase C)
  for (int ccd = blockIdx.x; ccd < B; ccd += gridDim.x) {
    __syncthreads();
    factor_diag(Lf + ccd * NN, dinv + (int64_t)ccd * nblk * NBK * NBK, status + ccd, N, 0, min(NBK, N), sa, sb, rinv);
  }
  bool ok = grid_sync_bounded(bar, &flag);
  for (int k = 0; ok && k < nblk; ++k) {
    const int kb = k * NBK, nb = min(NBK, N - kb), rem = N - kb - nb;
    if (rem <= 0) break;   // uniform: the last block has no panel
    // (B) panels, 32-row tiles: X = A inv(L_kk)^T; thread (row tid / 8, columns tid % 8 + 8 m)
    const int T = (rem + NBK - 1) / NBK;
    for (int item = blockIdx.x; item < B * T; item += gridDim.x) {
      const int ccd = item / T, r0 = kb + nb + (item % T) * NBK;
      double* l = Lf + ccd * NN;
      const double* iv = dinv + ((int64_t)ccd * nblk + k) * NBK * NBK;
      __syncthreads();
      for (int e = tid; e < NBK * NBK; e += blockDim.x) {
        const int i = e / NBK, c = e % NBK;
        sb[i][c] = __ldcg(iv + e);
        sa[i][c] = (r0 + i < N && c < nb) ? __ldcg(l + (int64_t)(r0 + i) * N + kb + c) : 0.0;
      }
      __syncthreads();
      const int i = tid >> 3, c0 = tid & 7;
      double out[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int c = c0 + 8 * m;
        double s0 = 0.0, s1 = 0.0;
        for (int t = 0; t + 1 <= c; t += 2) {
          s0 += sa[i][t] * sb[c][t];
          s1 += sa[i][t + 1] * sb[c][t + 1];
        }
        if ((c & 1) == 0) s0 += sa[i][c] * sb[c][c];
        out[m] = s0 + s1;
      }
      __syncthreads();
#pragma unroll
      for (int m = 0; m < 4; ++m) sa[i][c0 + 8 * m] = out[m];
      __syncthreads();
      for (int e = tid; e < NBK * NBK; e += blockDim.x) {
        const int ii = e / NBK, c = e % NBK;
        if (r0 + ii < N && c < nb) l[(int64_t)(r0 + ii) * N + kb + c] = sa[ii][c];
      }
    }
    if (!(ok = grid_sync_bounded(bar, &flag))) break;
    // (C) trailing update of the lower tiles; the CTA holding tile (0, 0), the
    // next diagonal block, factors it right after its update
    const int ntile = T * (T + 1) / 2;
    const int r0 = kb + nb;
    for (int item = blockIdx.x; item < B * ntile; item += gridDim.x) {
      const int ccd = item / ntile;
      int t = item % ntile, bi = 0;
      while (t > bi) { t -= bi + 1; ++bi; }
      const int bj = t;
      const int i0 = r0 + bi * NBK, j0 = r0 + bj * NBK;
      double* l = Lf + ccd * NN;
      __syncthreads();
      for (int e = tid; e < NBK * NBK; e += blockDim.x) {
        const int i = e / NBK, c = e % NBK;
        sa[i][c] = (i0 + i < N && c < nb) ? __ldcg(l + (int64_t)(i0 + i) * N + kb + c) : 0.0;
        sb[i][c] = (j0 + i < N && c < nb) ? __ldcg(l + (int64_t)(j0 + i) * N + kb + c) : 0.0;
      }
      __syncthreads();
      for (int e = tid; e < NBK * NBK; e += blockDim.x) {
        const int i = e / NBK, j = e % NBK;
        const int gi = i0 + i, gj = j0 + j;
        if (gi >= N || gj >= N || gj > gi) continue;
        double s0 = 0.0, s1 = 0.0;
#pragma unroll 8
        for (int c = 0; c < NBK; c += 2) {
          s0 += sa[i][c] * sb[j][c];
          s1 += sa[i][c + 1] * sb[j][c + 1];
        }
        l[(int64_t)gi * N + gj] = __ldcg(l + (int64_t)gi * N + gj) - (s0 + s1);
      }
      if (bi == 0) {   // tile (0, 0): the diagonal block of step k + 1 is final
        __syncthreads();
        factor_diag(l, dinv + ((int64_t)ccd * nblk + k + 1) * NBK * NBK, status + ccd, N, r0, min(NBK, N - r0),
                    sa, sb, rinv);
      }
    }
    ok = grid_sync_bounded(bar, &flag);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && ((volatile GridBar*)bar)->abort != 0u)
    for (int c = 0; c < B; ++c) atomicOr(&status[c], 4);
}

// x = D_s (L L^T)^-1 D_s rhs, one CTA per CCD, blocked substitution with the
// inverted diagonal blocks: each block of unknowns is a 32 x 32 product by one
// warp, the coupling to the remaining unknowns is applied by all threads.
__global__ void __launch_bounds__(1024)
k_chol_solve(const double* __restrict__ Lf, const double* __restrict__ dinv, const double* __restrict__ scale,
             const double* __restrict__ rhs, double* __restrict__ x, int N, int* __restrict__ status) {
  extern __shared__ double sh[];   // y[N]
  __shared__ double ld[NBK][NBK + 1];
  const int ccd = blockIdx.x;
  const int nblk = (N + NBK - 1) / NBK;
  const double* l = Lf + (int64_t)ccd * N * N;
  const double* s = scale + (int64_t)ccd * N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < N; i += blockDim.x) sh[i] = rhs[(int64_t)ccd * N + i] * s[i];
  // forward: L y = r
  for (int bi = 0; bi < nblk; ++bi) {
    const int jb = bi * NBK, nb = min(NBK, N - jb);
    const double* inv = dinv + ((int64_t)ccd * nblk + bi) * NBK * NBK;
    for (int e = threadIdx.x; e < NBK * NBK; e += blockDim.x) ld[e / NBK][e % NBK] = inv[e];
    __syncthreads();
    if (warp == 0) {
      const double v = lane < nb ? sh[jb + lane] : 0.0;
      double y0 = 0.0, y1 = 0.0;
#pragma unroll
      for (int t = 0; t < NBK; t += 2) {
        y0 += ld[lane][t] * __shfl_sync(0xffffffffu, v, t);
        y1 += ld[lane][t + 1] * __shfl_sync(0xffffffffu, v, t + 1);
      }
      if (lane < nb) sh[jb + lane] = y0 + y1;
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
    const int jb = bi * NBK, nb = min(NBK, N - jb);
    const double* inv = dinv + ((int64_t)ccd * nblk + bi) * NBK * NBK;
    for (int e = threadIdx.x; e < NBK * NBK; e += blockDim.x) ld[e / NBK][e % NBK] = inv[e];
    __syncthreads();
    if (warp == 0) {
      const double v = lane < nb ? sh[jb + lane] : 0.0;
      double z0 = 0.0, z1 = 0.0;
#pragma unroll
      for (int t = 0; t < NBK; t += 2) {
        z0 += ld[t][lane] * __shfl_sync(0xffffffffu, v, t);
        z1 += ld[t + 1][lane] * __shfl_sync(0xffffffffu, v, t + 1);
      }
      if (lane < nb) sh[jb + lane] = z0 + z1;
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

static CprMap cpr_map(const sfft_plan_s* p) {
  CprMap m;
  m.on = p->cpr ? 1 : 0;
  m.NK = p->NK;
  m.jc = (p->d.L * p->d.L - 1) / 2;
  m.nkc = (p->d.L * p->d.L - 1) * p->NK;
  return m;
}

cudaError_t launch_cholesky(const sfft_plan_s* p, const double* A, void* ws) {
  const int N = p->Nsol, B = p->d.batch;
  double* Lf = ws_at<double>(ws, p->lfac);
  double* scale = ws_at<double>(ws, p->scale);
  int* status = ws_at<int>(ws, p->status);
  double* dinv = ws_at<double>(ws, p->dinv);
  GridBar* bar = ws_at<GridBar>(ws, p->gbar);
  dim3 gi(64, B);
  k_chol_init<<<gi, 256, 0, p->stream>>>(A, Lf, scale, status, p->N, N, cpr_map(p));
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), p->stream);
  if (e != cudaSuccess) return e;
  // every CTA of the cooperative grid must be resident at once
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_coop, 256, 0);
  const int T0 = (N - NBK + NBK - 1) / NBK;
  const int want = std::max(B, B * T0 * (T0 + 1) / 2);
  const int grid = std::max(1, std::min(want, sms * std::max(per_sm, 1)));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = p->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_chol_coop, Lf, dinv, status, N, B, bar);
  p->nlaunch += 2;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_chol_solve(const sfft_plan_s* p, const double* rhs, double* x, void* ws) {
  const int N = p->Nsol;
  const size_t smem = sizeof(double) * N;
  cudaFuncSetAttribute(k_chol_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_chol_solve<<<p->d.batch, 1024, smem, p->stream>>>(ws_at<double>(ws, p->lfac), ws_at<double>(ws, p->dinv),
                                                      ws_at<double>(ws, p->scale), rhs, x, N,
                                                      ws_at<int>(ws, p->status));
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_theta_finish(const sfft_plan_s* p, const double* x, double* theta_off, bool add) {
  const int64_t n = (int64_t)p->N * p->d.batch;
  k_theta_finish<<<(int)((n + 255) / 256), 256, 0, p->stream>>>(x, theta_off, p->N, p->d.batch, add ? 1 : 0);
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_cpr_rhs(const sfft_plan_s* p, const double* b, double* out) {
  dim3 grid((p->Nsol + 255) / 256, p->d.batch);
  k_cpr_rhs<<<grid, 256, 0, p->stream>>>(b, out, p->N, p->Nsol, cpr_map(p));
  p->nlaunch += 1;
  return cudaGetLastError();
}

cudaError_t launch_cpr_expand(const sfft_plan_s* p, const double* x, double* theta_off, bool add) {
  dim3 grid((p->N + 255) / 256, p->d.batch);
  k_cpr_expand<<<grid, 256, 0, p->stream>>>(x, theta_off, p->N, p->Nsol, cpr_map(p), add ? 1 : 0);
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
