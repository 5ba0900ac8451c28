// C ABI: plan construction, workspace layout, contraction job tables and the
// entry points that enqueue the kernels on the plan's stream.
#include <math.h>
#include <string.h>

#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "plan.h"

using namespace sfft;

static thread_local std::string g_last_error;

void sfft::set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

static sfft_status_t cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return SFFT_ERR_CUDA;
}
#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
  } while (0)

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ------------------------------------------------------------------ instrumentation
static bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
  return st != cudaStreamCaptureStatusNone;
}

static cudaEvent_t pool_event(sfft_plan_s* p) {
  if (!p->evpool.empty()) {
    cudaEvent_t e = p->evpool.back();
    p->evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Counts the kernels a phase enqueues and, when profiling, brackets it with events.
struct Phase {
  sfft_plan_s* p;
  int cls;
  int64_t n0;
  cudaEvent_t a = nullptr;
  Phase(sfft_plan_s* pp, int c) : p(pp), cls(c), n0(pp->nlaunch) {
    if (p->prof && !stream_capturing(p->stream)) {
      a = pool_event(p);
      if (a) cudaEventRecord(a, p->stream);
    }
  }
  ~Phase() {
    p->prof_launch[cls] += p->nlaunch - n0;
    if (a) {
      cudaEvent_t b = pool_event(p);
      if (b) {
        cudaEventRecord(b, p->stream);
        p->pending.push_back({cls, a, b});
      } else {
        p->evpool.push_back(a);
      }
    }
  }
};

static void add_region(Region& r, size_t& cursor, size_t bytes) {
  r.off = cursor;
  r.bytes = bytes;
  cursor = align256(cursor + bytes);
}

static int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

template <typename T2, typename R>
static void fill_twiddles(sfft_plan_s* p, std::vector<T2>& twM, std::vector<T2>& twN, std::vector<T2>& twD) {
  const double pi = 3.14159265358979323846;
  twM.resize((size_t)p->M);
  for (int j = 0; j < p->M; ++j) {
    const double ang = -2.0 * pi * (double)j / (double)p->M;
    twM[j] = T2{(R)cos(ang), (R)sin(ang)};
  }
  twN.resize(p->M);
  for (int k = 0; k < p->M; ++k) {
    const double ang = -2.0 * pi * (double)k / (double)p->Nf;
    twN[k] = T2{(R)cos(ang), (R)sin(ang)};
  }
  twD.resize(p->Nf);
  for (int j = 0; j < p->Nf; ++j) {
    const double ang = 2.0 * pi * (double)j / (double)p->Nf;
    twD[j] = T2{(R)cos(ang), (R)sin(ang)};
  }
}

static void build_layout(sfft_plan_s* p) {
  const int64_t H = p->d.H, W = p->d.W, B = p->d.batch, M = p->M;
  const size_t e = p->elem, c = 2 * p->elem;
  const size_t npx = (size_t)H * W;
  const size_t slab = (size_t)H * M * c;
  const int LL = p->d.L * p->d.L;
  size_t cur = 0;
  add_region(p->status, cur, sizeof(int) * B);
  add_region(p->sky, cur, sizeof(double) * 2 * B);
  add_region(p->skyacc, cur, sizeof(double) * 4 * B);
  add_region(p->good, cur, npx * B);
  add_region(p->gh, cur, npx * B);
  add_region(p->mfit, cur, npx * B);
  add_region(p->rowflag, cur, sizeof(int) * (size_t)p->rf_stride * B);
  add_region(p->rm, cur, npx * e * B);
  add_region(p->eimg, cur, npx * e * B);
  add_region(p->wspec, cur, slab * p->n_wa * B);
  add_region(p->uspec, cur, slab * (p->d.DK + 1) * B);
  add_region(p->rhat, cur, slab * B);
  add_region(p->phat, cur, slab * p->d_batch * p->ccd_group);
  add_region(p->gkk, cur, sizeof(double) * p->n_hd * LL * n_mono(p->DM_KK) * B);
  add_region(p->gkb, cur, sizeof(double) * LL * n_mono(p->DM_KB) * B);
  add_region(p->gbk, cur, sizeof(double) * LL * n_mono(p->DM_bK) * B);
  add_region(p->mom_bb, cur, sizeof(double) * n_mono(p->DM_BB) * B);
  add_region(p->mom_b, cur, sizeof(double) * n_mono(p->d.DB) * B);
  add_region(p->lfac, cur, sizeof(double) * p->N * p->N * B);
  add_region(p->scale, cur, sizeof(double) * p->N * B);
  add_region(p->dinv, cur, sizeof(double) * 1024 * ((p->N + 31) / 32) * B);   // inverted 32 x 32 diagonal blocks
  add_region(p->gbar, cur, 64);                                               // grid barrier of the factorisation
  // substitutions: the y and x vectors, read by other CTAs as they appear
  add_region(p->swave, cur, sizeof(double) * 2 * p->N * B);
  add_region(p->vec, cur, sizeof(double) * 4 * p->N * B);
  // lane-per-difference contraction: k-slot products C[k][d_local][u_y][32] per CCD of a group
  add_region(p->cbuf, cur, p->dl ? sizeof(float) * (size_t)p->M * p->d_batch * p->d.L * 32 * p->ccd_group : 0);
  add_region(p->theta_off, cur, sizeof(double) * p->N * B);
  p->ws_bytes = cur;
}

static void build_jobs(sfft_plan_s* p) {
  const int L = p->d.L, w = p->w, B = p->d.batch, H = p->d.H;
  const int LL = L * L;
  const int MU = p->fp64 ? 6 : 11;
  const size_t slab = (size_t)H * p->M * 2 * p->elem;
  auto push_split = [&](CJob j) {
    for (int lo = j.uy_lo; lo <= j.uy_hi; lo += MU) {
      CJob q = j;
      q.uy_lo = lo;
      q.uy_hi = std::min(j.uy_hi, lo + MU - 1);
      p->h_jobs.push_back(q);
    }
  };
  p->h_jobs.clear();
  p->kk_first.clear();
  p->kk_count.clear();
  for (int d0 = 0; d0 < p->n_hd; d0 += p->d_batch) {
    const int nd = std::min(p->d_batch, p->n_hd - d0);
    p->kk_first.push_back((int)p->h_jobs.size());
    for (int ccd = 0; ccd < B; ++ccd)
      for (int i = 0; i < nd; ++i) {
        const int2 d = p->dlist[d0 + i];
        CJob j;
        j.probe = (int64_t)(p->phat.off + ((size_t)(ccd % p->ccd_group) * p->d_batch + i) * slab);
        j.wts = (int64_t)(p->wspec.off + (size_t)ccd * p->n_wa * slab);
        j.out = (int64_t)(p->gkk.off + sizeof(double) * ((size_t)ccd * p->n_hd + d0 + i) * LL * n_mono(p->DM_KK));
        j.rowflag = (int64_t)(p->rowflag.off + sizeof(int) * (size_t)ccd * p->rf_stride);
        j.status = (int64_t)(p->status.off + sizeof(int) * (size_t)ccd);
        j.uy_lo = std::max(-w, d.x - w);
        j.uy_hi = std::min(w, d.x + w);
        j.ux_lo = std::max(-w, d.y - w);
        j.ux_hi = std::min(w, d.y + w);
        push_split(j);
      }
    p->kk_count.push_back((int)p->h_jobs.size() - p->kk_first.back());
  }
  p->kb_first = (int)p->h_jobs.size();
  for (int ccd = 0; ccd < B; ++ccd) {
    CJob j;
    j.probe = (int64_t)(p->rhat.off + (size_t)ccd * slab);
    j.wts = (int64_t)(p->wspec.off + (size_t)ccd * p->n_wa * slab);
    j.out = (int64_t)(p->gkb.off + sizeof(double) * (size_t)ccd * LL * n_mono(p->DM_KB));
    j.rowflag = (int64_t)(p->rowflag.off + sizeof(int) * (size_t)ccd * p->rf_stride);
    j.status = (int64_t)(p->status.off + sizeof(int) * (size_t)ccd);
    j.uy_lo = -w; j.uy_hi = w; j.ux_lo = -w; j.ux_hi = w;
    push_split(j);
  }
  p->kb_count = (int)p->h_jobs.size() - p->kb_first;
  p->bk_first = (int)p->h_jobs.size();
  for (int ccd = 0; ccd < B; ++ccd) {
    CJob j;
    j.probe = (int64_t)(p->rhat.off + (size_t)ccd * slab);
    j.wts = (int64_t)(p->uspec.off + (size_t)ccd * (p->d.DK + 1) * slab);
    j.out = (int64_t)(p->gbk.off + sizeof(double) * (size_t)ccd * LL * n_mono(p->DM_bK));
    j.rowflag = (int64_t)(p->rowflag.off + sizeof(int) * (size_t)ccd * p->rf_stride);
    j.status = (int64_t)(p->status.off + sizeof(int) * (size_t)ccd);
    j.uy_lo = -w; j.uy_hi = w; j.ux_lo = -w; j.ux_hi = w;
    push_split(j);
  }
  p->bk_count = (int)p->h_jobs.size() - p->bk_first;
}

// Pair lists and patterns of the tensor-core KK contraction: per d-batch the
// (d, u_y) pairs in difference order, cut greedily into patterns of at most
// NP pairs from at most max_nd differences whose staged probe rows (chunk +
// n_lag - 1 per difference) fit `cap`; one job per (CCD, pattern).
static void build_tc_jobs(sfft_plan_s* p, int NP, int chunk, int cap, int max_nd) {
  const int L = p->d.L, w = p->w, B = p->d.batch, H = p->d.H;
  const int LL = L * L;
  const size_t slab = (size_t)H * p->M * 2 * p->elem;
  p->tc_first.clear();
  p->tc_count.clear();
  p->h_tcjobs.clear();
  p->h_tcpairs.clear();
  p->h_tcdj.clear();
  for (int d0 = 0; d0 < p->n_hd; d0 += p->d_batch) {
    const int nd = std::min(p->d_batch, p->n_hd - d0);
    const int pair_base = (int)p->h_tcpairs.size();
    for (int i = 0; i < nd; ++i) {
      const int2 d = p->dlist[d0 + i];
      const int ulo = std::max(-w, d.x - w), uhi = std::min(w, d.x + w);
      const int xlo = std::max(-w, d.y - w), xhi = std::min(w, d.y + w);
      for (int u = ulo; u <= uhi; ++u) p->h_tcpairs.push_back(int4{i, u, xlo, xhi});
    }
    struct Pat { int pair0, npair, dj0, nd; };
    std::vector<Pat> pats;
    const int npairs = (int)p->h_tcpairs.size() - pair_base;
    int q = 0;
    while (q < npairs) {
      Pat pt{pair_base + q, 0, (int)p->h_tcdj.size(), 0};
      int rows = 0;
      while (q < npairs && pt.npair < NP) {
        const int4 e = p->h_tcpairs[pair_base + q];
        const bool new_d = pt.nd == 0 || p->h_tcdj.back().x != e.x;
        const int add = new_d ? chunk : 1;
        if (rows + add > cap || (new_d && pt.nd == max_nd)) break;
        if (new_d) {
          p->h_tcdj.push_back(int4{e.x, e.y, e.y, rows});
          ++pt.nd;
        } else {
          p->h_tcdj.back().z = e.y;
        }
        rows += add;
        ++pt.npair;
        ++q;
      }
      pats.push_back(pt);
    }
    p->tc_first.push_back((int)p->h_tcjobs.size());
    for (int ccd = 0; ccd < B; ++ccd)
      for (const Pat& pt : pats) {
        TcJob j;
        j.probe = (int64_t)(p->phat.off + (size_t)(ccd % p->ccd_group) * p->d_batch * slab);
        j.wts = (int64_t)(p->wspec.off + (size_t)ccd * p->n_wa * slab);
        j.out = (int64_t)(p->gkk.off + sizeof(double) * ((size_t)ccd * p->n_hd + d0) * LL * n_mono(p->DM_KK));
        j.status = (int64_t)(p->status.off + sizeof(int) * (size_t)ccd);
        j.pair0 = pt.pair0;
        j.npair = pt.npair;
        j.dj0 = pt.dj0;
        j.nd = pt.nd;
        j.zp = (ccd % p->ccd_group) * p->d_batch;
        j.zw = ccd * p->n_wa;
        p->h_tcjobs.push_back(j);
      }
    p->tc_count.push_back((int)p->h_tcjobs.size() - p->tc_first.back());
  }
}

// Jobs of the lane-per-difference tensor-core contraction: per d-batch and
// CCD, tiles of up to 128 consecutive differences, each with its u_y range
// (the union over its differences) cut into runs of at most kDlMaxU; and
// the (d_local, u_y, ux_lo, ux_hi) pairs whose lags k_lag_dft forms.
static void build_dl_jobs(sfft_plan_s* p) {
  const int w = p->w, B = p->d.batch, H = p->d.H;
  const size_t cb_ccd = sizeof(float) * (size_t)p->M * p->d_batch * p->d.L * 32;
  p->dl_first.clear();
  p->dl_count.clear();
  p->dlp_first.clear();
  p->dlp_count.clear();
  p->h_dljobs.clear();
  p->h_dlpairs.clear();
  for (int d0 = 0; d0 < p->n_hd; d0 += p->d_batch) {
    const int nd = std::min(p->d_batch, p->n_hd - d0);
    p->dlp_first.push_back((int)p->h_dlpairs.size());
    for (int i = 0; i < nd; ++i) {
      const int2 d = p->dlist[d0 + i];
      const int ulo = std::max(-w, d.x - w), uhi = std::min(w, d.x + w);
      const int xlo = std::max(-w, d.y - w), xhi = std::min(w, d.y + w);
      for (int u = ulo; u <= uhi; ++u) p->h_dlpairs.push_back(int4{i, u, xlo, xhi});
    }
    p->dlp_count.push_back((int)p->h_dlpairs.size() - p->dlp_first.back());
    p->dl_first.push_back((int)p->h_dljobs.size());
    for (int ccd = 0; ccd < B; ++ccd)
      for (int t0 = 0; t0 < nd; t0 += 128) {
        const int nl = std::min(128, nd - t0);
        int ulo = w, uhi = -w;
        for (int i = t0; i < t0 + nl; ++i) {
          const int2 d = p->dlist[d0 + i];
          ulo = std::min(ulo, std::max(-w, d.x - w));
          uhi = std::max(uhi, std::min(w, d.x + w));
        }
        const int nrun = (uhi - ulo + kDlMaxU) / kDlMaxU;
        {
          const int y_lo = w, y_hi = H - w;
          for (int r = 0; r < nrun; ++r) {
            // runs of near-equal length
            const int a = ulo + (uhi - ulo + 1) * r / nrun, b = ulo + (uhi - ulo + 1) * (r + 1) / nrun;
            DlJob j;
            j.cbuf = (int64_t)(p->cbuf.off + (size_t)(ccd % p->ccd_group) * cb_ccd);
            j.status = (int64_t)(p->status.off + sizeof(int) * (size_t)ccd);
            j.zp = (ccd % p->ccd_group) * p->d_batch;
            j.zw = ccd * p->n_wa;
            j.d_first = t0;
            j.nlanes = nl;
            j.u_lo = a;
            j.nu = b - a;
            j.y_lo = y_lo;
            j.y_hi = y_hi;
            p->h_dljobs.push_back(j);
          }
        }
      }
    p->dl_count.push_back((int)p->h_dljobs.size() - p->dl_first.back());
  }
}

// ------------------------------------------------------------------ device allocations
// Every device allocation of a plan (its tables, and the autotuner's
// temporary buffers) goes through plan_malloc / plan_free, which count the
// live ones.  For fault-injection tests, SFFT_FAIL_ALLOC=n in the environment
// makes the n-th allocation of each sfft_plan call fail (without calling
// cudaMalloc), as a full device would.
static std::atomic<long long> g_live_allocs{0};
static thread_local int g_plan_depth = 0;
static thread_local long long g_plan_allocs = 0;

cudaError_t sfft::plan_malloc(void** dst, size_t bytes) {
  *dst = nullptr;
  const long long n = ++g_plan_allocs;
  const char* env = getenv("SFFT_FAIL_ALLOC");
  if (env && *env && atoll(env) == n) {
    g_last_error = "injected device allocation failure (SFFT_FAIL_ALLOC=" + std::string(env) + ")";
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMalloc(dst, bytes ? bytes : 1);
  if (e == cudaSuccess) {
    ++g_live_allocs;
  } else {
    *dst = nullptr;
    g_last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    cudaGetLastError();   // a failed allocation must not poison later calls
  }
  return e;
}

void sfft::plan_free(void* ptr) {
  if (!ptr) return;
  cudaFree(ptr);
  --g_live_allocs;
}

extern "C" int64_t sfft_debug_live_allocations(void) { return (int64_t)g_live_allocs.load(); }

static void free_plan_device(sfft_plan_s* p) {
  plan_free(p->d_dljobs);
  plan_free(p->d_dlpairs);
  plan_free(p->d_tcjobs);
  plan_free(p->d_tcpairs);
  plan_free(p->d_tcdj);
  plan_free(p->twM);
  plan_free(p->twN);
  plan_free(p->twD);
  plan_free(p->ytab);
  plan_free(p->d_dlist);
  plan_free(p->d_hdidx);
  plan_free(p->d_jobs);
  p->d_dljobs = nullptr; p->d_dlpairs = nullptr; p->d_tcjobs = nullptr; p->d_tcpairs = nullptr;
  p->d_tcdj = nullptr; p->twM = p->twN = p->twD = p->ytab = nullptr;
  p->d_dlist = nullptr; p->d_hdidx = nullptr; p->d_jobs = nullptr;
  for (auto& kv : p->graphs) cudaGraphExecDestroy(kv.second);
  p->graphs.clear();
  for (auto& e : p->pending) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  p->pending.clear();
  for (auto e : p->evpool) cudaEventDestroy(e);
  p->evpool.clear();
}

template <typename T>
static sfft_status_t upload(void** dst, const std::vector<T>& v) {
  const size_t bytes = sizeof(T) * std::max<size_t>(v.size(), 1);
  if (plan_malloc(dst, bytes) != cudaSuccess) return SFFT_ERR_NOMEM;
  if (!v.empty()) CK(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return SFFT_OK;
}

static sfft_status_t plan_impl(const sfft_desc_t* desc, void* cuda_stream, sfft_plan_t* out);

extern "C" sfft_status_t sfft_plan(const sfft_desc_t* desc, void* cuda_stream, sfft_plan_t* out) {
  // allocations are numbered per outermost call (the autotuner plans inside)
  if (g_plan_depth++ == 0) g_plan_allocs = 0;
  const sfft_status_t st = plan_impl(desc, cuda_stream, out);
  --g_plan_depth;
  return st;
}

static sfft_status_t plan_impl(const sfft_desc_t* desc, void* cuda_stream, sfft_plan_t* out) {
  if (!desc || !out) return SFFT_ERR_ARG;
  *out = nullptr;
  const sfft_desc_t d = *desc;
  if (d.H <= 0 || d.W <= 0 || d.batch <= 0 || d.L <= 0) return SFFT_ERR_ARG;
  if (d.prec != SFFT_PREC_FP64 && d.prec != SFFT_PREC_MIXED) return SFFT_ERR_ARG;
  if (d.DK < 0 || d.DB < 0 || d.d_batch < 0 || d.rows_per_cta < 0 || d.ccd_group < 0) return SFFT_ERR_ARG;
  if (d.lag_parts < 0 || d.lag_parts > 3) return SFFT_ERR_ARG;
  if ((d.L & 1) == 0 || d.L > kMaxL) return SFFT_ERR_UNSUPPORTED;
  if (d.flags & ~(SFFT_FLAG_GRAPH | SFFT_FLAG_CONST_RATIO | SFFT_FLAG_FMA_CONTRACT | SFFT_FLAG_MMA_SYNC_CONTRACT |
                  SFFT_FLAG_PAIR_LANE_CONTRACT))
    return SFFT_ERR_ARG;
  if (d.DK > kMaxD || d.DB > kMaxD) return SFFT_ERR_UNSUPPORTED;
  if (d.H < d.L || d.W < d.L || d.W < 16 || d.W > 2048) return SFFT_ERR_UNSUPPORTED;

  sfft_plan_s* p = new (std::nothrow) sfft_plan_s();
  if (!p) return SFFT_ERR_NOMEM;
  p->d = d;
  p->stream = (cudaStream_t)cuda_stream;
  p->fp64 = (d.prec == SFFT_PREC_FP64);
  p->elem = p->fp64 ? 8 : 4;
  cudaGetDevice(&p->device);
  p->w = (d.L - 1) / 2;
  p->NK = n_mono(d.DK);
  p->NB = n_mono(d.DB);
  p->NKK = d.L * d.L * p->NK;
  p->N = p->NKK + p->NB;
  p->cpr = (d.flags & SFFT_FLAG_CONST_RATIO) != 0;
  p->Nsol = p->cpr ? (d.L * d.L - 1) * p->NK + 1 + p->NB : p->N;
  p->Nf = std::max(64, next_pow2(d.W));
  p->M = p->Nf / 2;
  p->N2 = p->M / 32;
  p->DM_KK = 2 * d.DK;
  p->DM_KB = d.DK + d.DB;
  p->DM_bK = d.DK;
  p->DM_BB = 2 * d.DB;
  p->n_wa = std::max(p->DM_KK, p->DM_KB) + 1;
  std::vector<int> hdidx((size_t)(2 * d.L - 1) * (2 * d.L - 1), -1);
  for (int dy = 0; dy < d.L; ++dy)
    for (int dx = -(d.L - 1); dx < d.L; ++dx)
      if (dy > 0 || dx >= 0) {
        hdidx[(size_t)(dy + d.L - 1) * (2 * d.L - 1) + (dx + d.L - 1)] = (int)p->dlist.size();
        p->dlist.push_back(int2{dy, dx});
      }
  p->n_hd = (int)p->dlist.size();
  const size_t slab = (size_t)d.H * p->M * 2 * p->elem;
  // product spectra of up to 64 GB per CCD pass (GB300: 288 GB of HBM3e).
  // The product-spectrum stage runs per group of CCDs with every difference
  // in one pass when one CCD's spectra fit (7.4 GB at 2048 x 4096), on the
  // same contraction engine as a single CCD; otherwise one CCD at a time with
  // as many differences as fit.  A group holds at most 32 GB of spectra: the
  // difference-lane contraction measured 3.47 / 3.33 / 3.30 / 3.30 ms per
  // CCD with groups of 1 / 2 / 3 / 4 CCDs, but 5.2 ms with 9 (67 GB).
  const size_t budget = size_t(64) << 30, group_budget = size_t(32) << 30;
  const int d_batch_max = (int)std::max<size_t>(1, std::min<size_t>(budget / slab, (size_t)p->n_hd));
  int tuned_db = 0, tuned_rows = 0, tuned_parts = 0;
  if (d.autotune && (d.d_batch == 0 || d.rows_per_cta == 0 || d.lag_parts == 0)) {
    const sfft_status_t ts = autotune_tiles(d, (cudaStream_t)cuda_stream, d_batch_max, &tuned_db, &tuned_rows,
                                            &tuned_parts, &p->tuned_ms);
    if (ts != SFFT_OK) {
      delete p;
      return ts;
    }
  }
  if (d.d_batch > 0) p->d_batch = std::min(d.d_batch, p->n_hd);
  else p->d_batch = tuned_db > 0 ? std::min(tuned_db, p->n_hd) : d_batch_max;
  if (d.rows_per_cta > 0) p->rows_per_cta = d.rows_per_cta;
  else p->rows_per_cta = tuned_rows > 0 ? tuned_rows : std::min(d.H, 1024);
  p->ccd_group =
      (int)std::max<size_t>(1, std::min<size_t>(group_budget / (slab * (size_t)p->d_batch), (size_t)d.batch));
  if (d.ccd_group > 0) p->ccd_group = std::min(d.ccd_group, d.batch);
  if (d.lag_parts > 0) p->csplit = d.lag_parts;
  else p->csplit = tuned_parts > 0 ? tuned_parts : 2;
  if (p->fp64) p->csplit = 2;
  // row flags are bulk-copied in 16-byte aligned runs of up to 20 ints past a chunk start
  p->rf_stride = ((d.H + 32) + 63) / 64 * 64;
  p->tc = !p->fp64 && !(d.flags & SFFT_FLAG_FMA_CONTRACT);
  p->umma = p->tc && !(d.flags & SFFT_FLAG_MMA_SYNC_CONTRACT);
  // one lane per difference needs two whole k-slots per CTA and difference
  // batches that fill most of the 128 lanes
  p->dl = p->umma && !(d.flags & SFFT_FLAG_PAIR_LANE_CONTRACT) && p->M % 16 == 0 && d.H >= 32 &&
          p->d_batch >= std::min(p->n_hd, 96);
  p->tc_rows = d.H;
  build_layout(p);
  build_jobs(p);
  if (p->dl) build_dl_jobs(p);
  if (p->umma) build_tc_jobs(p, kUmmaPairs, 1, 1 << 30, kUmmaMaxDiffs);
  else if (p->tc) build_tc_jobs(p, 8 * kTcNT, kTcChunk, kTcRowCap, 1 << 30);

  // yt(y)^b for b = 0..4 per row, FP64 on the host, stored in the path's precision
  std::vector<double> ypow((size_t)d.H * 8, 0.0);
  for (int y = 0; y < d.H; ++y) {
    const double yt = 2.0 * y / (double)(d.H > 1 ? d.H - 1 : 1) - 1.0;
    double pw = 1.0;
    for (int b = 0; b < 5; ++b) { ypow[(size_t)y * 8 + b] = pw; pw *= yt; }
  }

  sfft_status_t st = SFFT_OK;
  if (p->fp64) {
    std::vector<double2> a, b, c;
    fill_twiddles<double2, double>(p, a, b, c);
    if (st == SFFT_OK) st = upload(&p->twM, a);
    if (st == SFFT_OK) st = upload(&p->twN, b);
    if (st == SFFT_OK) st = upload(&p->twD, c);
    if (st == SFFT_OK) st = upload(&p->ytab, ypow);
  } else {
    std::vector<float2> a, b, c;
    fill_twiddles<float2, float>(p, a, b, c);
    if (st == SFFT_OK) st = upload(&p->twM, a);
    if (st == SFFT_OK) st = upload(&p->twN, b);
    if (st == SFFT_OK) st = upload(&p->twD, c);
    // FP32 rows hold each power twice, (yt^0, yt^0, yt^1, yt^1, ...), so that the
    // contraction loads them as ready-made operand pairs of the packed FP32 FMA
    std::vector<float> ypf((size_t)d.H * 16, 0.0f);
    for (int y = 0; y < d.H; ++y)
      for (int b = 0; b < 5; ++b) ypf[(size_t)y * 16 + 2 * b] = ypf[(size_t)y * 16 + 2 * b + 1] = (float)ypow[(size_t)y * 8 + b];
    if (st == SFFT_OK) st = upload(&p->ytab, ypf);
  }
  if (st == SFFT_OK) st = upload((void**)&p->d_dlist, p->dlist);
  if (st == SFFT_OK) st = upload((void**)&p->d_hdidx, hdidx);
  if (st == SFFT_OK) st = upload((void**)&p->d_jobs, p->h_jobs);
  if (st == SFFT_OK && p->tc) st = upload((void**)&p->d_tcjobs, p->h_tcjobs);
  if (st == SFFT_OK && p->tc) st = upload((void**)&p->d_tcpairs, p->h_tcpairs);
  if (st == SFFT_OK && p->tc) st = upload((void**)&p->d_tcdj, p->h_tcdj);
  if (st == SFFT_OK && p->dl) st = upload((void**)&p->d_dljobs, p->h_dljobs);
  if (st == SFFT_OK && p->dl) st = upload((void**)&p->d_dlpairs, p->h_dlpairs);
  if (st != SFFT_OK) {
    free_plan_device(p);
    delete p;
    return st;
  }
  *out = p;
  return SFFT_OK;
}

extern "C" void sfft_plan_destroy(sfft_plan_t p) {
  if (!p) return;
  free_plan_device(p);
  delete p;
}

extern "C" sfft_status_t sfft_plan_set_stream(sfft_plan_t p, void* s) {
  if (!p) return SFFT_ERR_ARG;
  p->stream = (cudaStream_t)s;
  return SFFT_OK;
}

extern "C" sfft_status_t sfft_plan_set_wait_limit(sfft_plan_t p, int32_t tries) {
  if (!p) return SFFT_ERR_ARG;
  p->bar_spin_limit = tries < 0 ? (1 << 24) : tries;
  return SFFT_OK;
}

extern "C" int64_t sfft_num_unknowns(sfft_plan_t p) { return p ? p->N : -1; }
extern "C" size_t sfft_workspace_bytes(sfft_plan_t p) { return p ? p->ws_bytes : 0; }
extern "C" int32_t sfft_plan_engine(sfft_plan_t p) {
  if (!p) return -1;
  if (p->fp64) return 0;
  if (!p->tc) return 1;
  if (!p->umma) return 2;
  return p->dl ? 4 : 3;
}
extern "C" int32_t sfft_plan_ccd_group(sfft_plan_t p) { return p ? p->ccd_group : -1; }

extern "C" sfft_status_t sfft_plan_tiles(sfft_plan_t p, int32_t* o) {
  if (!p || !o) return SFFT_ERR_ARG;
  o[0] = p->d_batch; o[1] = p->rows_per_cta; o[2] = p->csplit;
  return SFFT_OK;
}

static bool aligned(const void* ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

static sfft_status_t build_normal_impl(sfft_plan_t p, const float* R, const float* S, const uint8_t* bad,
                                       const double* sky, double* A, double* b, void* ws) {
  cudaStream_t st = p->stream;
  {
    Phase ph(p, SFFT_PROF_PREP);
    CK(cudaMemsetAsync(ws_at<char>(ws, p->status), 0, p->status.bytes, st));
    CK(launch_sky(p, R, S, bad, sky, ws));
    CK(launch_prep(p, R, S, bad, ws));
    CK(launch_moments(p, S, nullptr, false, ws));
  }
  {
    Phase ph(p, SFFT_PROF_FFT_WEIGHTS);
    CK(launch_rfft_rm(p, ws));
    CK(launch_rfft_weights(p, nullptr, nullptr, 0, p->n_wa, ws_at<char>(ws, p->wspec), p->n_wa, ws));
    CK(launch_rfft_weights(p, S, nullptr, 0, p->d.DK + 1, ws_at<char>(ws, p->uspec), p->d.DK + 1, ws));
  }
  {
    Phase ph(p, SFFT_PROF_CONTRACT_RK);
    CK(cudaMemsetAsync(ws_at<char>(ws, p->gkk), 0, p->gkk.bytes, st));
    CK(cudaMemsetAsync(ws_at<char>(ws, p->gkb), 0, p->gkb.bytes, st));
    CK(cudaMemsetAsync(ws_at<char>(ws, p->gbk), 0, p->gbk.bytes, st));
    CK(launch_contract(p, p->DM_KB, p->kb_first, p->kb_count, p->rows_per_cta, p->csplit, ws));
    CK(launch_contract(p, p->DM_bK, p->bk_first, p->bk_count, p->rows_per_cta, p->csplit, ws));
  }
  // product spectra and their contraction: per group of ccd_group CCDs, per d-batch
  const int B = p->d.batch, G = p->ccd_group;
  for (int c0 = 0; c0 < B; c0 += G) {
    const int nc = std::min(G, B - c0);
    for (size_t ib = 0; ib < p->kk_first.size(); ++ib) {
      const int d0 = (int)ib * p->d_batch;
      const int nd = std::min(p->d_batch, p->n_hd - d0);
      // the d-batch's KK jobs are ordered CCD-major with the same count per CCD
      const int jpc = p->kk_count[ib] / B;
      const int kj0 = p->kk_first[ib] + c0 * jpc, kjn = nc * jpc;
      {
        Phase ph(p, SFFT_PROF_FFT_PROD);
        CK(launch_rfft_prod(p, c0, nc, d0, nd, ws));
      }
      {
        Phase ph(p, SFFT_PROF_CONTRACT_KK);
        if (p->tc) {
          if (p->dl) CK(launch_contract_dlane(p, (int)ib, c0, nc, ws));
          else CK(p->umma ? launch_contract_umma(p, (int)ib, c0, nc, ws) : launch_contract_tc(p, (int)ib, c0, nc, ws));
        } else {
          CK(launch_contract(p, p->DM_KK, kj0, kjn, p->rows_per_cta, p->csplit, ws));
        }
      }
      if (p->tc) {
        Phase ph(p, SFFT_PROF_LAG_DFT);
        if (p->dl) CK(launch_lag_dft(p, (int)ib, c0, nc, ws));
        CK(launch_contract_slot0(p, p->DM_KK, kj0, kjn, ws));
      }
    }
  }
  {
    Phase ph(p, SFFT_PROF_SCATTER);
    CK(launch_scatter(p, A, b, ws, false, nullptr));
  }
  return SFFT_OK;
}

static sfft_status_t solve_impl(sfft_plan_t p, const double* A, const double* b, double* theta, int32_t refine,
                                const float* R, const float* S, int32_t* info, void* ws) {
  double* vec = ws_at<double>(ws, p->vec);
  const size_t NBt = (size_t)p->N * p->d.batch;
  double* rhs = vec;
  double* x = vec + NBt;
  double* toff = ws_at<double>(ws, p->theta_off);
  // constant-ratio fit: right-hand sides projected to, and solutions expanded
  // from, the constrained basis (vec's third and fourth quarters)
  double* rhs_c = vec + 2 * NBt;
  double* x_c = vec + 3 * NBt;
  auto solve_rhs = [&](const double* r, bool add) -> sfft_status_t {
    if (p->cpr) {
      CK(launch_cpr_rhs(p, r, rhs_c));
      CK(launch_chol_solve(p, rhs_c, x_c, ws));
      CK(launch_cpr_expand(p, x_c, toff, add));
    } else {
      CK(launch_chol_solve(p, r, x, ws));
      CK(launch_theta_finish(p, x, toff, add));
    }
    return SFFT_OK;
  };
  {
    Phase ph(p, SFFT_PROF_SOLVE);
    CK(launch_cholesky(p, A, ws));
    const sfft_status_t s0 = solve_rhs(b, false);
    if (s0 != SFFT_OK) return s0;
    if (!p->fp64 && refine == 0) {
      // the FP32 factor's solution, refined once against the FP64 system
      // (the image-space steps below refine it otherwise)
      CK(launch_residual(p, A, b, toff, rhs));
      const sfft_status_t s1 = solve_rhs(rhs, true);
      if (s1 != SFFT_OK) return s1;
    }
  }
  for (int r = 0; r < refine; ++r) {
    void* e = ws_at<char>(ws, p->eimg);
    {
      Phase ph(p, SFFT_PROF_APPLY);
      CK(launch_apply(p, R, S, toff, nullptr, nullptr, e, true, ws));
    }
    {
      Phase ph(p, SFFT_PROF_FFT_WEIGHTS);
      CK(launch_rfft_weights(p, nullptr, e, 0, p->d.DK + 1, ws_at<char>(ws, p->uspec), p->d.DK + 1, ws));
    }
    {
      Phase ph(p, SFFT_PROF_CONTRACT_RK);
      CK(cudaMemsetAsync(ws_at<char>(ws, p->gbk), 0, p->gbk.bytes, p->stream));
      CK(launch_contract(p, p->DM_bK, p->bk_first, p->bk_count, p->rows_per_cta, p->csplit, ws));
    }
    {
      Phase ph(p, SFFT_PROF_PREP);
      CK(launch_moments(p, nullptr, e, true, ws));
    }
    {
      Phase ph(p, SFFT_PROF_SCATTER);
      CK(launch_scatter(p, nullptr, nullptr, ws, true, rhs));
    }
    {
      Phase ph(p, SFFT_PROF_SOLVE);
      const sfft_status_t s1 = solve_rhs(rhs, true);
      if (s1 != SFFT_OK) return s1;
    }
  }
  {
    Phase ph(p, SFFT_PROF_SOLVE);
    CK(launch_theta_to_orig(p, toff, theta, ws));
    if (info) CK(launch_info(p, info, ws));
  }
  return SFFT_OK;
}

static sfft_status_t apply_impl(sfft_plan_t p, const float* R, const float* S, const double* theta,
                                const double* sky, float* D, void* ws) {
  double* toff = ws_at<double>(ws, p->theta_off);
  Phase ph(p, SFFT_PROF_APPLY);
  CK(launch_theta_to_off(p, theta, sky, toff, ws));
  CK(launch_apply(p, R, S, toff, sky, D, nullptr, false, ws));
  return SFFT_OK;
}

static sfft_status_t check_common(sfft_plan_t p, const void* R, const void* S, const void* ws) {
  if (!p || !R || !S || !ws) return SFFT_ERR_ARG;
  if (!aligned(ws, 256)) return SFFT_ERR_ARG;
  if (!aligned(R, 4) || !aligned(S, 4)) return SFFT_ERR_ARG;
  return SFFT_OK;
}

extern "C" sfft_status_t sfft_build_normal(sfft_plan_t p, const float* R, const float* S, const uint8_t* bad,
                                           const double* sky, double* A, double* b, void* ws) {
  sfft_status_t s = check_common(p, R, S, ws);
  if (s != SFFT_OK) return s;
  if (!A || !b) return SFFT_ERR_ARG;
  return build_normal_impl(p, R, S, bad, sky, A, b, ws);
}

extern "C" sfft_status_t sfft_solve(sfft_plan_t p, const double* A, const double* b, double* theta,
                                    int32_t refine_steps, const float* R, const float* S, const uint8_t* bad,
                                    int32_t* info, void* ws) {
  (void)bad;
  if (!p || !A || !b || !theta || !ws || refine_steps < 0) return SFFT_ERR_ARG;
  if (refine_steps > 0 && (!R || !S)) return SFFT_ERR_ARG;
  return solve_impl(p, A, b, theta, refine_steps, R, S, info, ws);
}

extern "C" sfft_status_t sfft_apply(sfft_plan_t p, const float* R, const float* S, const double* theta,
                                    const double* sky, float* D, void* ws) {
  sfft_status_t s = check_common(p, R, S, ws);
  if (s != SFFT_OK) return s;
  if (!theta || !D) return SFFT_ERR_ARG;
  return apply_impl(p, R, S, theta, sky, D, ws);
}

static sfft_status_t subtract_enqueue(sfft_plan_t p, const float* R, const float* S, const uint8_t* bad,
                                      const double* sky, int32_t refine, double* A, double* b, double* theta,
                                      int32_t* info, float* D, void* ws) {
  sfft_status_t s = build_normal_impl(p, R, S, bad, sky, A, b, ws);
  if (s != SFFT_OK) return s;
  s = solve_impl(p, A, b, theta, refine, R, S, info, ws);
  if (s != SFFT_OK) return s;
  return apply_impl(p, R, S, theta, nullptr, D, ws);
}

extern "C" sfft_status_t sfft_subtract(sfft_plan_t p, const float* R, const float* S, const uint8_t* bad,
                                       const double* sky, int32_t refine_steps, double* A, double* b,
                                       double* theta, int32_t* info, float* D, void* ws) {
  sfft_status_t s = check_common(p, R, S, ws);
  if (s != SFFT_OK) return s;
  if (!A || !b || !theta || !D || refine_steps < 0) return SFFT_ERR_ARG;
  if (!(p->d.flags & SFFT_FLAG_GRAPH) || p->stream == nullptr)
    return subtract_enqueue(p, R, S, bad, sky, refine_steps, A, b, theta, info, D, ws);
  std::vector<uintptr_t> key = {(uintptr_t)R, (uintptr_t)S, (uintptr_t)bad, (uintptr_t)sky, (uintptr_t)refine_steps,
                                (uintptr_t)A, (uintptr_t)b, (uintptr_t)theta, (uintptr_t)info, (uintptr_t)D,
                                (uintptr_t)ws};
  auto it = p->graphs.find(key);
  if (it == p->graphs.end()) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    sfft_status_t es = subtract_enqueue(p, R, S, bad, sky, refine_steps, A, b, theta, info, D, ws);
    cudaError_t ce = cudaStreamEndCapture(p->stream, &g);
    if (es != SFFT_OK) { if (g) cudaGraphDestroy(g); return es; }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    ce = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
    it = p->graphs.emplace(key, ex).first;
  }
  CK(cudaGraphLaunch(it->second, p->stream));
  return SFFT_OK;
}

extern "C" sfft_status_t sfft_kernel_at(sfft_plan_t p, const double* theta, double x, double y, double* K) {
  if (!p || !theta || !K) return SFFT_ERR_ARG;
  CK(launch_kernel_at(p, theta, x, y, K));
  return SFFT_OK;
}

extern "C" sfft_status_t sfft_profile_enable(sfft_plan_t p, int32_t enable) {
  if (!p) return SFFT_ERR_ARG;
  p->prof = enable != 0;
  return SFFT_OK;
}

extern "C" sfft_status_t sfft_profile_read(sfft_plan_t p, double* ms, int64_t* launches, int32_t reset) {
  if (!p) return SFFT_ERR_ARG;
  if (!p->pending.empty()) {
    CK(cudaStreamSynchronize(p->stream));
    for (auto& e : p->pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) p->prof_ms[e.cls] += t;
      p->evpool.push_back(e.a);
      p->evpool.push_back(e.b);
    }
    p->pending.clear();
  }
  for (int i = 0; i < SFFT_PROF_N; ++i) {
    if (ms) ms[i] = p->prof_ms[i];
    if (launches) launches[i] = p->prof_launch[i];
    if (reset) { p->prof_ms[i] = 0.0; p->prof_launch[i] = 0; }
  }
  return SFFT_OK;
}

extern "C" const char* sfft_status_str(sfft_status_t s) {
  switch (s) {
    case SFFT_OK: return "ok";
    case SFFT_ERR_ARG: return "invalid argument";
    case SFFT_ERR_CUDA: return "CUDA error";
    case SFFT_ERR_NOMEM: return "out of memory";
    case SFFT_ERR_SINGULAR: return "normal matrix not positive definite";
    case SFFT_ERR_NONFINITE: return "non-finite normal matrix or solution";
    case SFFT_ERR_TIMEOUT: return "bounded device wait timed out";
    case SFFT_ERR_UNSUPPORTED: return "unsupported shape or degree";
  }
  return "unknown status";
}

extern "C" const char* sfft_last_error(void) { return g_last_error.c_str(); }
