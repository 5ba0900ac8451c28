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
// diagonal blocks (one cooperative launch, blocks handed between CTAs by
// flags), theta = D_s y.
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

// scale = diag(A_s)^-1/2 and the diagonal's status flags, a thread per row.
// A_s is the solved system: A itself (row stride N = Ns) or T A T^T (size Ns).
__global__ void k_chol_scale(const double* __restrict__ A, double* __restrict__ scale, int* __restrict__ status,
                             int N, int Ns, CprMap m) {
  const int ccd = blockIdx.y;
  const double* a = A + ccd * (int64_t)N * N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Ns; i += gridDim.x * blockDim.x) {
    const double d = cpr_entry(a, N, m, i, i);
    if (!isfinite(d)) atomicOr(&status[ccd], 2);
    else if (!(d > 0.0)) atomicOr(&status[ccd], 1);
    scale[(int64_t)ccd * Ns + i] = d > 0.0 ? rsqrt(d) : 0.0;
  }
}

// Lf (lower) = D_s A_s D_s with D_s = diag(scale): a CTA per row (strided),
// a thread per column.  Two FP64 products per element; the reciprocal
// square roots (a few dozen FP64 operations each on a pipe that retires
// about two per SM per clock) are formed once per row by k_chol_scale.
template <typename T>
__global__ void __launch_bounds__(256)
k_chol_init(const double* __restrict__ A, T* __restrict__ Lf, const double* __restrict__ scale,
            int* __restrict__ status, int N, int Ns, CprMap m) {
  const int ccd = blockIdx.y;
  const double* a = A + ccd * (int64_t)N * N;
  T* l = Lf + ccd * (int64_t)Ns * Ns;
  const double* s = scale + (int64_t)ccd * Ns;
  for (int i = blockIdx.x; i < Ns; i += gridDim.x) {
    const double si = s[i];
    for (int j = threadIdx.x; j <= i; j += blockDim.x) {
      const double v = cpr_entry(a, N, m, i, j);
      if (!isfinite(v)) atomicOr(&status[ccd], 2);
      l[(int64_t)i * Ns + j] = (T)(v * si * s[j]);
    }
  }
}

// ---------------------------------------------------------------- persistent blocked Cholesky
// One cooperative launch (one CTA per SM for a few CCDs) factors every CCD's
// matrix.  For each 32-column block k: (B) the CTAs take 8-row pieces of the
// panels below the diagonal blocks and solve X L_kk^T = A by substitution
// (a warp per row, a lane per column); (C) they take 8 x 32 pieces of the
// trailing lower triangles and subtract P_i P_j^T, while one CTA per CCD
// updates the next diagonal block in shared memory and factors it
// (look-ahead).  GB300 retires about two FP64 FMAs per SM per clock, so the
// pieces are small enough to spread each step over every SM, and the chain
// from one diagonal block to the next is kept short: the block factor takes
// one barrier per column and maps the threads onto the elements each column
// step touches, and the inverses of the diagonal factors, which only the
// substitutions need, are formed after the last step, all blocks at once.
// The phases are separated by a grid-wide barrier whose waits are bounded:
// a barrier that gives up (or sees another CTA give up) flags every CCD with
// bit 4 and the kernel returns.  Data written by other CTAs is read with
// L2-coherent loads (ld.global.cg).
struct GridBar { unsigned count, gen, abort, pad; };

constexpr int kBarSpin = 1 << 24;   // x >= 64 ns per try: about a second (the default wait limit)
constexpr int PRW = 8;              // rows per piece of the panel and trailing updates
constexpr int NTRI = NBK * (NBK + 1) / 2;

__device__ bool grid_sync_bounded(GridBar* bar, int* flag_sh, int spin_limit) {
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
        if (*vab != 0u || it >= spin_limit) { ok = false; break; }
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

template <typename T>
struct CholSmem {
  T blk[NBK][NBK + 1];   // diagonal block, or the rows of a piece
  T aux[NBK][NBK + 1];   // a diagonal factor, panel rows, or an inverse
  T pinv[NBK], prs[NBK], dgl[NBK];   // per pivot d: 1 / d, 1 / sqrt(d), sqrt(d)
  unsigned char ti[NTRI], tj[NTRI];       // e -> (i, j), j <= i, e = i (i + 1) / 2 + j
  int flag;
};

// Pivot c: a non-positive or non-finite d is replaced by 1 and reported in
// the CCD's status word.
__device__ __forceinline__ double rsq(double d) { return rsqrt(d); }
__device__ __forceinline__ float rsq(float d) { return rsqrtf(d); }

template <typename T>
__device__ __forceinline__ void set_pivot(CholSmem<T>& S, int c, T d0, int* st) {
  const bool bad = !(d0 > T(0)) || !isfinite(d0);
  if (bad) atomicOr(st, isfinite(d0) ? 1 : 2);
  const T d = bad ? T(1) : d0;
  const T r = rsq(d);
  S.pinv[c] = r * r;
  S.prs[c] = r;
  S.dgl[c] = d * r;
}

// Factor S.blk (lower, identity past the block's size) in place: right-
// looking on the unscaled Schur complement, a_ij -= a_ic a_jc / d_c for
// c < j <= i, one barrier per column (the thread that updates the next
// diagonal element forms its pivot at once), then l_ij = a_ij / sqrt(d_j).
template <typename T>
__device__ void factor_block(CholSmem<T>& S, int* st) {
  const int tid = threadIdx.x;
  if (tid == 0) set_pivot(S, 0, S.blk[0][0], st);
  __syncthreads();
  for (int c = 0; c < NBK - 1; ++c) {
    const T p = S.pinv[c];
    const int m = NBK - 1 - c;
    for (int e = tid; e < m * (m + 1) / 2; e += blockDim.x) {
      const int i = c + 1 + S.ti[e], j = c + 1 + S.tj[e];
      const T v = S.blk[i][j] - S.blk[i][c] * S.blk[j][c] * p;
      S.blk[i][j] = v;
      if (e == 0) set_pivot(S, c + 1, v, st);   // (i, j) = (c + 1, c + 1)
    }
    __syncthreads();
  }
  for (int e = tid; e < NTRI; e += blockDim.x) {
    const int i = S.ti[e], j = S.tj[e];
    S.blk[i][j] = i == j ? S.dgl[j] : S.blk[i][j] * S.prs[j];
  }
  __syncthreads();
}

// S.aux = inverse of the lower factor in S.blk (L X = I by row elimination:
// row t is final once scaled, then removed below).
template <typename T>
__device__ void invert_block(CholSmem<T>& S) {
  const int tid = threadIdx.x;
  for (int e = tid; e < NBK * (NBK + 1); e += blockDim.x) {
    const int i = e / (NBK + 1), j = e % (NBK + 1);
    S.aux[i][j] = i == j ? T(1) : T(0);
  }
  if (tid < NBK) S.pinv[tid] = T(1) / S.blk[tid][tid];
  __syncthreads();
  for (int t = 0; t < NBK; ++t) {
    if (tid <= t) S.aux[t][tid] *= S.pinv[t];
    __syncthreads();
    const int w = t + 1, n = (NBK - 1 - t) * w;
    for (int e = tid; e < n; e += blockDim.x) {
      const int i = t + 1 + e / w, j = e % w;
      S.aux[i][j] -= S.blk[i][t] * S.aux[t][j];
    }
    __syncthreads();
  }
}

// S.blk <- the factored diagonal block at rows/columns [r0, r0 + nb) of l
// (identity past nb)
template <typename T>
__device__ void load_block(const T* __restrict__ l, int N, int r0, int nb, T (*dst)[NBK + 1]) {
  for (int e = threadIdx.x; e < NBK * NBK; e += blockDim.x) {
    const int i = e / NBK, j = e % NBK;
    dst[i][j] = (i < nb && j <= i) ? __ldcg(l + (int64_t)(r0 + i) * N + r0 + j) : (i == j ? T(1) : T(0));
  }
}

template <typename T>
__device__ void store_block(const CholSmem<T>& S, T* __restrict__ l, int N, int r0, int nb) {
  for (int e = threadIdx.x; e < NTRI; e += blockDim.x) {
    const int i = S.ti[e], j = S.tj[e];
    if (i < nb) l[(int64_t)(r0 + i) * N + r0 + j] = S.blk[i][j];
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_chol_coop(T* __restrict__ Lf, T* __restrict__ dinv, int* __restrict__ status, int N, int B,
            GridBar* __restrict__ bar, int spin_limit) {
  __shared__ CholSmem<T> S;
  const int nblk = (N + NBK - 1) / NBK;
  const int64_t NN = (int64_t)N * N;
  const int tid = threadIdx.x, G = gridDim.x;
  const int warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < NTRI; e += blockDim.x) {
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    S.ti[e] = (unsigned char)i;
    S.tj[e] = (unsigned char)(e - i * (i + 1) / 2);
  }
  // the first diagonal block of every CCD; later ones are factored as soon
  // as their last trailing update lands (look-ahead inside phase C)
  for (int ccd = blockIdx.x; ccd < B; ccd += G) {
    __syncthreads();
    load_block(Lf + ccd * NN, N, 0, min(NBK, N), S.blk);
    __syncthreads();
    factor_block(S, status + ccd);
    store_block(S, Lf + ccd * NN, N, 0, min(NBK, N));
  }
  bool ok = grid_sync_bounded(bar, &S.flag, spin_limit);
  for (int k = 0; ok && k < nblk; ++k) {
    const int kb = k * NBK, nb = min(NBK, N - kb), rem = N - kb - nb;
    if (rem <= 0) break;   // uniform: the last block has no panel
    const int TB = (rem + NBK - 1) / NBK;   // block rows below the diagonal block
    const int r0 = kb + nb;
    // (B) panel pieces: X L_kk^T = A, warp = row of the piece, lane = column
    for (int item = blockIdx.x; item < B * TB * (NBK / PRW); item += G) {
      const int ccd = item / (TB * (NBK / PRW)), pc = item % (TB * (NBK / PRW));
      const int p0 = r0 + pc * PRW;
      T* l = Lf + ccd * NN;
      __syncthreads();
      load_block(l, N, kb, nb, S.aux);
      for (int e = tid; e < PRW * NBK; e += blockDim.x) {
        const int i = e / NBK, c = e % NBK;
        S.blk[i][c] = (p0 + i < N && c < nb) ? __ldcg(l + (int64_t)(p0 + i) * N + kb + c) : T(0);
      }
      __syncthreads();
      if (warp < PRW) {
        const T rd = T(1) / S.aux[lane][lane];
        T acc = S.blk[warp][lane], x = T(0);
#pragma unroll 4
        for (int t = 0; t < NBK; ++t) {
          if (lane == t) x = acc * rd;
          const T xt = __shfl_sync(0xffffffffu, x, t);
          if (lane > t) acc -= xt * S.aux[lane][t];
        }
        if (p0 + warp < N && lane < nb) l[(int64_t)(p0 + warp) * N + kb + lane] = x;
      }
    }
    if (!(ok = grid_sync_bounded(bar, &S.flag, spin_limit))) break;
    // (C) the next diagonal block of every CCD (one CTA each: update and
    // factor), then 8 x 32 pieces of the other trailing tiles
    const int ntile = TB * (TB + 1) / 2;
    const int npiece = (ntile - 1) * (NBK / PRW);
    for (int item = blockIdx.x; item < B + B * npiece; item += G) {
      __syncthreads();
      if (item < B) {
        const int ccd = item, nb2 = min(NBK, rem);
        T* l = Lf + ccd * NN;
        for (int e = tid; e < NBK * NBK; e += blockDim.x) {
          const int i = e / NBK, c = e % NBK;
          S.aux[i][c] = (i < nb2 && c < nb) ? __ldcg(l + (int64_t)(r0 + i) * N + kb + c) : T(0);
        }
        __syncthreads();
        for (int e = tid; e < NTRI; e += blockDim.x) {
          const int i = S.ti[e], j = S.tj[e];
          T v = i == j ? T(1) : T(0);
          if (i < nb2) {
            T s0 = T(0), s1 = T(0);
#pragma unroll 8
            for (int c = 0; c < NBK; c += 2) {
              s0 += S.aux[i][c] * S.aux[j][c];
              s1 += S.aux[i][c + 1] * S.aux[j][c + 1];
            }
            v = __ldcg(l + (int64_t)(r0 + i) * N + r0 + j) - (s0 + s1);
          }
          S.blk[i][j] = v;
        }
        __syncthreads();
        factor_block(S, status + ccd);
        store_block(S, l, N, r0, nb2);
        continue;
      }
      const int q = item - B, ccd = q / npiece, pc = q % npiece;
      int t = 1 + pc / (NBK / PRW), bi = 0;
      while (t > bi) { t -= bi + 1; ++bi; }
      const int bj = t;
      const int i0 = r0 + bi * NBK + (pc % (NBK / PRW)) * PRW, j0 = r0 + bj * NBK;
      T* l = Lf + ccd * NN;
      for (int e = tid; e < NBK * NBK; e += blockDim.x) {
        const int j = e / NBK, c = e % NBK;
        S.aux[j][c] = (j0 + j < N && c < nb) ? __ldcg(l + (int64_t)(j0 + j) * N + kb + c) : T(0);
      }
      for (int e = tid; e < PRW * NBK; e += blockDim.x) {
        const int i = e / NBK, c = e % NBK;
        S.blk[i][c] = (i0 + i < N && c < nb) ? __ldcg(l + (int64_t)(i0 + i) * N + kb + c) : T(0);
      }
      __syncthreads();
      const int i = tid / NBK, j = tid % NBK;
      const int gi = i0 + i, gj = j0 + j;
      if (i < PRW && gi < N && gj < N && gj <= gi) {
        T s0 = T(0), s1 = T(0);
#pragma unroll 8
        for (int c = 0; c < NBK; c += 2) {
          s0 += S.blk[i][c] * S.aux[j][c];
          s1 += S.blk[i][c + 1] * S.aux[j][c + 1];
        }
        l[(int64_t)gi * N + gj] = __ldcg(l + (int64_t)gi * N + gj) - (s0 + s1);
      }
    }
    ok = grid_sync_bounded(bar, &S.flag, spin_limit);
  }
  // inverses of the diagonal factors for the substitutions, all at once
  for (int item = blockIdx.x; ok && item < B * nblk; item += G) {
    const int ccd = item / nblk, b = item % nblk, jb = b * NBK;
    __syncthreads();
    load_block(Lf + ccd * NN, N, jb, min(NBK, N - jb), S.blk);
    __syncthreads();
    invert_block(S);
    T* out = dinv + ((int64_t)ccd * nblk + b) * NBK * NBK;
    for (int e = tid; e < NBK * NBK; e += blockDim.x) out[e] = S.aux[e / NBK][e % NBK];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && ((volatile GridBar*)bar)->abort != 0u)
    for (int c = 0; c < B; ++c) atomicOr(&status[c], 4);
}

// ---------------------------------------------------------------- substitutions
// x = D_s (L L^T)^-1 D_s rhs in one cooperative launch.  The unknowns come
// in 32-blocks (CCD c, block b); item o = b B + c belongs to CTA o mod G.
// Forward (increasing o): the owner gathers r_b - sum_{j<b} L_bj y_j as the
// y_j appear, then publishes y_b = inv(L_bb) (...).  Backward (decreasing o):
// z_b = y_b - sum_{j>b} L_jb^T x_j, x_b = inv(L_bb)^T z_b.  The y and x
// buffers start as an all-ones bit pattern that no stored value has (a NaN
// result is stored as the canonical NaN), so a thread waits for exactly the
// values it reads, with the rows of L fetched before the wait.  Every item
// waits only on items of smaller order, each CTA takes its items in that
// order and the grid is co-resident, so the smallest unfinished item can
// always run.  The waits are bounded; one that gives up marks the CCDs
// (bit 4) and the CTA stops.
constexpr long long kUnset = -1ll;   // all bits set

template <typename T>
struct SolveSmem {
  T iv[NBK][NBK + 1];
  T v[NBK];
  T part[NBK][9];
  int fail;
};

__device__ __forceinline__ double publishable(double v) {
  return isnan(v) ? __longlong_as_double(0x7FF8000000000000ll) : v;
}
__device__ __forceinline__ float publishable(float v) { return isnan(v) ? __int_as_float(0x7FC00000) : v; }
__device__ __forceinline__ bool is_unset(double x) { return __double_as_longlong(x) == kUnset; }
__device__ __forceinline__ bool is_unset(float x) { return __float_as_int(x) == -1; }

template <typename T>
__device__ __forceinline__ bool wait_value(const T* p, T& v) {
  for (int it = 0; it < kBarSpin; ++it) {
    const T x = __ldcv(p);
    if (!is_unset(x)) {
      v = x;
      return true;
    }
    if (it > 16) __nanosleep(32);
  }
  return false;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_chol_solve(const T* __restrict__ Lf, const T* __restrict__ dinv, const double* __restrict__ scale,
             const double* __restrict__ rhs, double* __restrict__ x, int N, int B, T* __restrict__ ybuf,
             T* __restrict__ xbuf, int* __restrict__ status) {
  __shared__ SolveSmem<T> S;
  const int nblk = (N + NBK - 1) / NBK;
  const int nitem = nblk * B, G = gridDim.x;
  const int tid = threadIdx.x, row = tid >> 3, part = tid & 7;
  if (tid == 0) S.fail = 0;
  __syncthreads();
  bool alive = true, waited = true;
  // forward
  for (int o = blockIdx.x; alive && o < nitem; o += G) {
    const int b = o / B, ccd = o % B, jb = b * NBK, nb = min(NBK, N - jb);
    const T* l = Lf + (int64_t)ccd * N * N;
    const T* iv = dinv + ((int64_t)ccd * nblk + b) * NBK * NBK;
    for (int e = tid; e < NBK * NBK; e += blockDim.x) S.iv[e / NBK][e % NBK] = iv[e];
    T acc = T(0);   // thread (row, part): columns part + 8 m of every block j < b
    for (int j = 0; j < b && waited; ++j) {
      T lv[NBK / 8], yv[NBK / 8];
      const T* lr = l + (int64_t)(jb + min(row, nb - 1)) * N + j * NBK + part;
#pragma unroll
      for (int m = 0; m < NBK / 8; ++m) lv[m] = __ldcg(lr + 8 * m);
      const T* y = ybuf + (int64_t)ccd * N + j * NBK + part;
#pragma unroll
      for (int m = 0; m < NBK / 8; ++m) waited = waited && wait_value(y + 8 * m, yv[m]);
      if (waited && row < nb)
#pragma unroll
        for (int m = 0; m < NBK / 8; ++m) acc += lv[m] * yv[m];
    }
    if (!waited) S.fail = 1;
    S.part[row][part] = acc;
    __syncthreads();
    if (S.fail) { alive = false; break; }
    if (tid < NBK) {
      T s = T(0);
#pragma unroll
      for (int p = 0; p < 8; ++p) s += S.part[tid][p];
      S.v[tid] = tid < nb ? (T)(rhs[(int64_t)ccd * N + jb + tid] * scale[(int64_t)ccd * N + jb + tid]) - s : T(0);
    }
    __syncthreads();
    if (tid < nb) {
      T s0 = T(0), s1 = T(0);
#pragma unroll
      for (int t = 0; t < NBK; t += 2) {
        s0 += S.iv[tid][t] * S.v[t];
        s1 += S.iv[tid][t + 1] * S.v[t + 1];
      }
      ybuf[(int64_t)ccd * N + jb + tid] = publishable(s0 + s1);
    }
    __syncthreads();
  }
  // backward
  const int last = (alive && (int)blockIdx.x < nitem) ? (nitem - 1 - (int)blockIdx.x) / G * G + (int)blockIdx.x : -1;
  for (int o = last; alive && o >= 0; o -= G) {
    const int b = o / B, ccd = o % B, jb = b * NBK, nb = min(NBK, N - jb);
    const T* l = Lf + (int64_t)ccd * N * N;
    const T* iv = dinv + ((int64_t)ccd * nblk + b) * NBK * NBK;
    for (int e = tid; e < NBK * NBK; e += blockDim.x) S.iv[e / NBK][e % NBK] = iv[e];
    T acc = T(0);   // thread (column row, part): rows part + 8 m of every block j > b
    for (int j = nblk - 1; j > b && waited; --j) {
      const int nj = min(NBK, N - j * NBK);
      T lv[NBK / 8], xv[NBK / 8];
#pragma unroll
      for (int m = 0; m < NBK / 8; ++m) {
        const int r = min(part + 8 * m, nj - 1);
        lv[m] = __ldcg(l + (int64_t)(j * NBK + r) * N + jb + min(row, nb - 1));
      }
      const T* xs = xbuf + (int64_t)ccd * N + j * NBK;
#pragma unroll
      for (int m = 0; m < NBK / 8; ++m) {
        const int r = part + 8 * m;
        xv[m] = T(0);
        if (r < nj) waited = waited && wait_value(xs + r, xv[m]);
      }
      if (waited && row < nb)
#pragma unroll
        for (int m = 0; m < NBK / 8; ++m)
          if (part + 8 * m < nj) acc += lv[m] * xv[m];
    }
    if (!waited) S.fail = 1;
    S.part[row][part] = acc;
    __syncthreads();
    if (S.fail) { alive = false; break; }
    if (tid < NBK) {
      T s = T(0);
#pragma unroll
      for (int p = 0; p < 8; ++p) s += S.part[tid][p];
      S.v[tid] = tid < nb ? __ldcg(ybuf + (int64_t)ccd * N + jb + tid) - s : T(0);
    }
    __syncthreads();
    if (tid < nb) {
      T s0 = T(0), s1 = T(0);
#pragma unroll
      for (int t = 0; t < NBK; t += 2) {
        s0 += S.iv[t][tid] * S.v[t];
        s1 += S.iv[t + 1][tid] * S.v[t + 1];
      }
      const T z = s0 + s1;
      xbuf[(int64_t)ccd * N + jb + tid] = publishable(z);
      const double v = (double)z * scale[(int64_t)ccd * N + jb + tid];
      if (!isfinite(v)) atomicOr(&status[ccd], 2);
      x[(int64_t)ccd * N + jb + tid] = v;
    }
    __syncthreads();
  }
  if (!alive && tid == 0)
    for (int c = 0; c < B; ++c) atomicOr(&status[c], 4);
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
  // a wait that gave up leaves the normal matrix or the factor partly
  // unwritten, which then also looks singular or non-finite: the time-out is
  // the cause and is reported first
  info[c] = (s & 4) ? SFFT_ERR_TIMEOUT : ((s & 2) ? SFFT_ERR_NONFINITE : ((s & 1) ? SFFT_ERR_SINGULAR : SFFT_OK));
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

// Cooperative grid size: one CTA per SM for a few CCDs (the FP64 pipe of an
// SM is shared by its CTAs, and a smaller grid makes the grid-wide barriers
// cheaper); for a batch of 8 or more, as many as fit, to hide load latency.
// CTAs of a cooperative grid: at most `want`, all co-resident; one per SM
// for a small batch (`single` per SM, when they fit), as many as fit for 8+ CCDs
static int coop_grid(const void* fn, int want, int batch, int single = 1) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0);
  if (per_sm < 1) return 1;
  return std::max(1, std::min(want, sms * (batch >= 8 ? per_sm : std::min(per_sm, single))));
}

static cudaError_t launch_coop(const void* fn, int grid, cudaStream_t s, void** args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// The FP64 path factors and substitutes in FP64.  The mixed path factors the
// Jacobi-scaled matrix in FP32 (its condition number is a few hundred on the
// DECam-shaped pairs, so the FP32 factor's relative error on theta is about
// 5e-6) and every solution it enters is refined against the FP64 system: by
// the image-space refinement steps, whose right-hand side is the projection
// of the residual image (b - A theta), or, without them, by one normal-
// equations residual step (launch_residual).
template <typename T>
static cudaError_t cholesky_T(const sfft_plan_s* p, const double* A, void* ws) {
  int N = p->Nsol, B = p->d.batch;
  T* Lf = ws_at<T>(ws, p->lfac);
  double* scale = ws_at<double>(ws, p->scale);
  int* status = ws_at<int>(ws, p->status);
  T* dinv = ws_at<T>(ws, p->dinv);
  GridBar* bar = ws_at<GridBar>(ws, p->gbar);
  k_chol_scale<<<dim3((N + 255) / 256, B), 256, 0, p->stream>>>(A, scale, status, p->N, N, cpr_map(p));
  k_chol_init<T><<<dim3(std::min(N, 1024), B), 256, 0, p->stream>>>(A, Lf, scale, status, p->N, N, cpr_map(p));
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), p->stream);
  if (e != cudaSuccess) return e;
  // every CTA of the cooperative grid must be resident at once
  const int T0 = (N - NBK + NBK - 1) / NBK;
  const int want = std::max(B, B + B * std::max(T0 * (T0 + 1) / 2 - 1, 1) * (NBK / PRW));
  // FP32: three CTAs per SM shorten each block step's pieces (solve phase
  // 0.622 ms, against 0.637 with two and 0.69 with one); one per SM stays
  // better for the FP64 pipe
  const int grid = coop_grid((const void*)k_chol_coop<T>, want, B, sizeof(T) == 4 ? 3 : 1);
  int spin = p->bar_spin_limit;
  void* args[] = {&Lf, &dinv, &status, &N, &B, &bar, &spin};
  e = launch_coop((const void*)k_chol_coop<T>, grid, p->stream, args);
  p->nlaunch += 3;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_cholesky(const sfft_plan_s* p, const double* A, void* ws) {
  return p->fp64 ? cholesky_T<double>(p, A, ws) : cholesky_T<float>(p, A, ws);
}

template <typename T>
static cudaError_t chol_solve_T(const sfft_plan_s* p, const double* rhs, double* x, void* ws) {
  int N = p->Nsol, B = p->d.batch;
  const int nitem = ((N + NBK - 1) / NBK) * B;
  T* Lf = ws_at<T>(ws, p->lfac);
  T* dinv = ws_at<T>(ws, p->dinv);
  double* scale = ws_at<double>(ws, p->scale);
  T* ybuf = ws_at<T>(ws, p->swave);
  T* xbuf = ybuf + (size_t)p->N * B;
  int* status = ws_at<int>(ws, p->status);
  // y and x start unset (all bits one)
  cudaError_t e = cudaMemsetAsync(ybuf, 0xFF, sizeof(T) * 2 * (size_t)p->N * B, p->stream);
  if (e != cudaSuccess) return e;
  const int grid = coop_grid((const void*)k_chol_solve<T>, nitem, B);
  void* args[] = {&Lf, &dinv, &scale, &rhs, &x, &N, &B, &ybuf, &xbuf, &status};
  e = launch_coop((const void*)k_chol_solve<T>, grid, p->stream, args);
  p->nlaunch += 1;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_chol_solve(const sfft_plan_s* p, const double* rhs, double* x, void* ws) {
  return p->fp64 ? chol_solve_T<double>(p, rhs, x, ws) : chol_solve_T<float>(p, rhs, x, ws);
}

// r = b - A theta for every CCD (FP64; A full, N x N row-major): a warp per row
__global__ void __launch_bounds__(256)
k_residual(const double* __restrict__ A, const double* __restrict__ b, const double* __restrict__ theta,
           double* __restrict__ r, int N) {
  const int ccd = blockIdx.y, lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= N) return;   // whole warps
  const double* a = A + ((int64_t)ccd * N + row) * N;
  const double* t = theta + (int64_t)ccd * N;
  double s0 = 0.0, s1 = 0.0;
  int c = lane;
  for (; c + 32 < N; c += 64) {
    s0 += a[c] * t[c];
    s1 += a[c + 32] * t[c + 32];
  }
  if (c < N) s0 += a[c] * t[c];
  const double s = warp_sum(s0 + s1);
  if (lane == 0) r[(int64_t)ccd * N + row] = b[(int64_t)ccd * N + row] - s;
}

cudaError_t launch_residual(const sfft_plan_s* p, const double* A, const double* b, const double* theta_off,
                            double* r) {
  dim3 grid((p->N + 7) / 8, p->d.batch);
  k_residual<<<grid, 256, 0, p->stream>>>(A, b, theta_off, r, p->N);
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
