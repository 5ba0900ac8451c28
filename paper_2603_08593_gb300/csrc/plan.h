// Host-side plan object, workspace layout and kernel launcher declarations.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "sfft.h"

namespace sfft {

// One contraction job: correlate the weight spectra at workspace offset
// `wts` (a-indexed, stride H*M) against the probe spectrum at offset `probe`
// for lags u_y in [uy_lo, uy_hi], u_x in [ux_lo, ux_hi]; results accumulate
// (FP64) into out[(uy+w)][(ux+w)][m] at offset `out`.  Offsets are bytes from
// the workspace base so that job tables are built once per plan.
struct CJob {
  int64_t probe, wts, out, rowflag, status;
  int uy_lo, uy_hi, ux_lo, ux_hi;
};

struct Region { size_t off = 0, bytes = 0; };

// One CTA row of the tensor-core KK contraction (kernels_contract_tc.cu): the
// pairs [pair0, pair0 + npair) of the pair table (int4 (d_local, u_y, ux_lo,
// ux_hi), d_local within the d-batch) and the differences [dj0, dj0 + nd) of
// the pattern table (int4 (d_local, u_lo, u_hi, first staged row)).
struct TcJob {
  int64_t probe, wts, out, status;   // byte offsets: slab of d_local = 0, weight spectra, G of d_local = 0, status
  int pair0, npair, dj0, nd;
  int zp, zw;                        // the CCD's first product / weight spectrum in the batch-wide tensor maps
};
constexpr int kTcKT = 8;         // k-slots per CTA (one warp each)
constexpr int kTcNT = 8;         // 8-column tiles per warp: up to 64 (d, u_y) pairs per CTA
constexpr int kTcChunk = 32;     // weight rows per stage
constexpr int kTcRowCap = 448;   // staged probe rows per stage: sum over differences of (chunk + n_lag - 1)
// tcgen05 kernel (kernels_contract_umma.cu): 128 pairs per CTA (the MMA's M)
// drawn from at most 16 differences
constexpr int kUmmaKT = 8;
constexpr int kUmmaChunk = 32;
constexpr int kUmmaPairs = 128;
constexpr int kUmmaMaxDiffs = 16;
// tcgen05 kernel with one lane per difference (kernels_contract_dlane.cu):
// one CTA per (two k-slots, tile of up to 128 differences, up to kDlMaxU
// consecutive u_y); its accumulators go to C[k][d_local][u_y][32]
struct DlJob {
  int64_t cbuf, status;   // byte offsets: the CCD's C buffer of the d-batch, status
  int zp, zw;             // the CCD's first product / weight spectrum in the batch-wide tensor maps
  int d_first, nlanes;    // the tile: differences [d_first, d_first + nlanes) of the d-batch
  int u_lo, nu;           // u_y = u_lo .. u_lo + nu - 1
  int y_lo, y_hi;         // weight rows [y_lo, y_hi): the band [w, H - w)
};
constexpr int kDlChunk = 16;
constexpr int kDlMaxU = 6;

}  // namespace sfft

struct sfft_plan_s {
  sfft_desc_t d{};
  cudaStream_t stream = nullptr;
  bool fp64 = false;
  int device = 0;
  int w = 0, NK = 0, NB = 0, NKK = 0, N = 0;
  bool cpr = false;                   // constant photometric ratio: solve in the constrained basis
  int Nsol = 0;                       // unknowns of the solved system: N, or (L^2 - 1) N_K + 1 + N_B
  int Nf = 0, M = 0, N2 = 0;
  int DM_KK = 0, DM_KB = 0, DM_bK = 0, DM_BB = 0;
  int n_wa = 0;                       // weight spectra a = 0 .. n_wa-1
  int n_hd = 0;                       // half-plane differences
  std::vector<int2> dlist;            // (dy, dx) per half-plane difference
  int d_batch = 0, rows_per_cta = 0, csplit = 2;   // csplit: lag parts per (k-slot, group) in the contraction
  int ccd_group = 1;                  // CCDs whose product spectra of one d-batch are held at once
  bool tc = false;                    // KK contraction on the tensor cores (FP32 path)
  bool umma = false;                  // ... with tcgen05 (else mma.sync)
  bool dl = false;                    // ... with one tensor-memory lane per difference (else per (d, u_y) pair)
  int tc_rows = 0;                    // weight rows per CTA of the tensor-core contraction
  double tuned_ms = 0.0;              // autotuned build_normal time per CCD (0: not tuned)
  int bar_spin_limit = 1 << 24;       // tries of the factorisation's grid-barrier wait (about a second)
  size_t elem = 4;                    // sizeof(T)
  // plan-owned constant device tables
  void* twM = nullptr;                // c_t [M]       exp(-2 pi i j / M)
  void* twN = nullptr;                // c_t [M]       exp(-2 pi i k / Nf)
  void* twD = nullptr;                // c_t [Nf]      (cos, sin)(2 pi j / Nf)
  void* ytab = nullptr;               // 64 B per row: yt(y)^b, b = 0..4, as double [8] (FP64 path) or as
                                      // duplicated pairs float [16] (FP32 path); zero padded
  int rf_stride = 0;                  // ints per CCD in the row-flag array (padded, multiple of 64)
  int2* d_dlist = nullptr;            // device copy of dlist
  int* d_hdidx = nullptr;             // [(2L-1)][(2L-1)] -> half-plane index or -1
  sfft::CJob* d_jobs = nullptr;       // job table (device), built at plan time
  std::vector<sfft::CJob> h_jobs;
  // job table sections: KK jobs of d-batch i start at kk_first[i]
  std::vector<int> kk_first, kk_count;
  int kb_first = 0, kb_count = 0, bk_first = 0, bk_count = 0;
  // tensor-core KK contraction: jobs of d-batch i start at tc_first[i]
  std::vector<int> tc_first, tc_count;
  std::vector<sfft::TcJob> h_tcjobs;
  std::vector<int4> h_tcpairs, h_tcdj;
  sfft::TcJob* d_tcjobs = nullptr;
  int4* d_tcpairs = nullptr;
  int4* d_tcdj = nullptr;
  // lane-per-difference engine: jobs and (d_local, u_y, ux_lo, ux_hi) pairs of d-batch i
  std::vector<int> dl_first, dl_count, dlp_first, dlp_count;
  std::vector<sfft::DlJob> h_dljobs;
  std::vector<int4> h_dlpairs;
  sfft::DlJob* d_dljobs = nullptr;
  int4* d_dlpairs = nullptr;
  // workspace regions (per-CCD strides where noted)
  sfft::Region sky, skyacc, good, gh, mfit, rowflag, rm, wspec, uspec, rhat, phat, gkk, gkb, gbk,
      mom_bb, mom_b, eimg, lfac, scale, dinv, gbar, swave, vec, theta_off, status, cbuf;
  size_t ws_bytes = 0;
  // graph cache for sfft_subtract
  std::map<std::vector<uintptr_t>, cudaGraphExec_t> graphs;
  // instrumentation: kernel launches (incremented by the launchers) and per-phase event timing
  mutable int64_t nlaunch = 0;
  bool prof = false;
  struct PendingEv { int cls; cudaEvent_t a, b; };
  std::vector<PendingEv> pending;
  std::vector<cudaEvent_t> evpool;
  double prof_ms[SFFT_PROF_N] = {};
  int64_t prof_launch[SFFT_PROF_N] = {};
};

namespace sfft {

// kernels_*.cu launchers; all enqueue on p->stream and return cudaGetLastError()
cudaError_t launch_sky(const sfft_plan_s* p, const float* R, const float* S, const uint8_t* bad,
                       const double* sky_in, void* ws);
cudaError_t launch_prep(const sfft_plan_s* p, const float* R, const float* S, const uint8_t* bad, void* ws);
cudaError_t launch_moments(const sfft_plan_s* p, const float* S, const void* eimg, bool resid, void* ws);
cudaError_t launch_rfft_rm(const sfft_plan_s* p, void* ws);
cudaError_t launch_rfft_weights(const sfft_plan_s* p, const float* S, const void* eimg, int a0, int na,
                                void* out, int nslab, void* ws);
// The product-spectrum stage runs per group of ccd_group CCDs: c0 is the
// group's first CCD, nc its size; product spectra and k-slot products are
// indexed within the group, everything else by the CCD's batch index.
cudaError_t launch_rfft_prod(const sfft_plan_s* p, int c0, int nc, int d0, int nd, void* ws);
cudaError_t launch_contract(const sfft_plan_s* p, int DM, int job0, int njobs, int rows_per_cta, int lag_parts,
                            void* ws);
cudaError_t launch_contract_tc(const sfft_plan_s* p, int batch_index, int c0, int nc, void* ws);
cudaError_t launch_contract_umma(const sfft_plan_s* p, int batch_index, int c0, int nc, void* ws);
cudaError_t launch_contract_dlane(const sfft_plan_s* p, int batch_index, int c0, int nc, void* ws);
cudaError_t launch_lag_dft(const sfft_plan_s* p, int batch_index, int c0, int nc, void* ws);
cudaError_t launch_contract_slot0(const sfft_plan_s* p, int DM, int job0, int njobs, void* ws);
cudaError_t launch_scatter(const sfft_plan_s* p, double* A, double* b, void* ws, bool rhs_only, double* rhs_out);
cudaError_t launch_cholesky(const sfft_plan_s* p, const double* A, void* ws);
cudaError_t launch_chol_solve(const sfft_plan_s* p, const double* rhs, double* x, void* ws);
cudaError_t launch_residual(const sfft_plan_s* p, const double* A, const double* b, const double* theta_off,
                            double* r);
cudaError_t launch_theta_finish(const sfft_plan_s* p, const double* x, double* theta_off, bool add);
cudaError_t launch_cpr_rhs(const sfft_plan_s* p, const double* b, double* out);
cudaError_t launch_cpr_expand(const sfft_plan_s* p, const double* x, double* theta_off, bool add);
cudaError_t launch_theta_to_orig(const sfft_plan_s* p, const double* theta_off, double* theta, void* ws);
cudaError_t launch_theta_to_off(const sfft_plan_s* p, const double* theta, const double* sky, double* theta_off, void* ws);
cudaError_t launch_apply(const sfft_plan_s* p, const float* R, const float* S, const double* theta_off,
                         const double* sky, float* D, void* eimg, bool resid, void* ws);
cudaError_t launch_info(const sfft_plan_s* p, int32_t* info, void* ws);
cudaError_t launch_kernel_at(const sfft_plan_s* p, const double* theta, double x, double y, double* K);

// Plan-free launchers (explicit shapes and stream) used by the allocation-free entry point.
cudaError_t launch_theta_units_raw(cudaStream_t s, const double* src, double* dst, const double* sky, int L, int NK,
                                   int NB, int batch, int to_orig);
cudaError_t launch_apply_raw(cudaStream_t s, bool fp64, const float* R, const float* S, const double* theta_off,
                             const double* sky, float* D, int H, int W, int L, int DK, int DB, int batch);
void set_last_error(const char* msg);
// Device allocations of plans and the autotuner (counted; see api.cu).
cudaError_t plan_malloc(void** dst, size_t bytes);
void plan_free(void* ptr);
// Times candidate (d_batch, rows_per_cta) on synthetic data (autotune.cu).
sfft_status_t autotune_tiles(const sfft_desc_t& d, cudaStream_t s, int d_batch_max, int* d_batch, int* rows_per_cta,
                             int* lag_parts, double* ms_per_ccd);

template <typename T> inline T* ws_at(void* ws, const Region& r) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + r.off);
}

}  // namespace sfft
