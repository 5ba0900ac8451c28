// Plan-time autotuning of the normal-matrix assembly's tile shape.
//
// Candidates are the number of kernel-offset differences per product/FFT pass
// (d_batch: the memory-budget maximum and its half), the rows of one
// contraction partial sum (rows_per_cta: 256 .. 2048, at most H) and the lag
// parts per contraction k-slot (2 or 3, FP32 path).  Each
// candidate builds a temporary plan of the same shape with min(batch, 2) CCDs,
// runs sfft_build_normal on synthetic images (every pixel good, so every row
// carries work) once to warm up and twice timed with CUDA events, and the
// fastest per-CCD time wins.  Results are kept per process, keyed by the
// descriptor, and appended to the file named by SFFT_AUTOTUNE_CACHE (one line
// "key d_batch rows_per_cta lag_parts ms") when that variable is set; a later process
// reads them back instead of timing again.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "plan.h"

namespace sfft {
namespace {

struct Tuned { int d_batch, rows_per_cta, lag_parts; double ms; };

std::mutex g_mu;
std::map<std::string, Tuned> g_cache;
bool g_loaded = false;

std::string tune_key(const sfft_desc_t& d, int device) {
  char buf[160];
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, device);
  snprintf(buf, sizeof(buf), "v3_sm%d%d_%dSM_H%d_W%d_L%d_DK%d_DB%d_B%d_P%d", prop.major, prop.minor,
           prop.multiProcessorCount, d.H, d.W, d.L, d.DK, d.DB, d.batch, d.prec);
  return buf;
}

void load_cache_file() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = getenv("SFFT_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[160];
  Tuned t{};
  while (fscanf(f, "%159s %d %d %d %lf", key, &t.d_batch, &t.rows_per_cta, &t.lag_parts, &t.ms) == 5) g_cache[key] = t;
  fclose(f);
}

void store(const std::string& key, const Tuned& t) {
  g_cache[key] = t;
  const char* path = getenv("SFFT_AUTOTUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), t.d_batch, t.rows_per_cta, t.lag_parts, t.ms);
  fclose(f);
}

// deterministic sky-like values: 1000 + a hash spread of +-64 ADU
__global__ void k_tune_fill(float* R, float* S, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const float u = (float)(h & 0xffff) * (1.0f / 65536.0f);
    R[i] = 1000.0f + 128.0f * (u - 0.5f);
    S[i] = 1000.0f + 128.0f * (0.5f - u);
  }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { plan_free(p); }
  bool alloc(size_t n) { return plan_malloc(&p, n) == cudaSuccess; }
};

// time one candidate; returns ms per CCD or a negative value on failure
double time_candidate(const sfft_desc_t& base, cudaStream_t s, int d_batch, int rows, int parts) {
  sfft_desc_t d = base;
  d.autotune = 0;
  d.flags = 0;
  d.batch = std::min(base.batch, 2);
  d.d_batch = d_batch;
  d.ccd_group = 0;
  d.rows_per_cta = rows;
  d.lag_parts = parts;
  sfft_plan_t p = nullptr;
  if (sfft_plan(&d, s, &p) != SFFT_OK) return -1.0;
  const int64_t npx = (int64_t)d.H * d.W * d.batch;
  const int64_t N = sfft_num_unknowns(p);
  DevBuf R, S, A, b, ws;
  double best = -1.0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (R.alloc(npx * 4) && S.alloc(npx * 4) && A.alloc((size_t)d.batch * N * N * 8) && b.alloc((size_t)d.batch * N * 8) &&
      ws.alloc(sfft_workspace_bytes(p)) && cudaEventCreate(&e0) == cudaSuccess &&
      cudaEventCreate(&e1) == cudaSuccess) {
    k_tune_fill<<<1024, 256, 0, s>>>((float*)R.p, (float*)S.p, npx);
    bool ok = sfft_build_normal(p, (const float*)R.p, (const float*)S.p, nullptr, nullptr, (double*)A.p,
                                (double*)b.p, ws.p) == SFFT_OK;
    for (int it = 0; ok && it < 2; ++it) {
      cudaEventRecord(e0, s);
      ok = sfft_build_normal(p, (const float*)R.p, (const float*)S.p, nullptr, nullptr, (double*)A.p,
                             (double*)b.p, ws.p) == SFFT_OK;
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        const double per = ms / d.batch;
        if (best < 0 || per < best) best = per;
      } else {
        ok = false;
      }
    }
    if (!ok) best = -1.0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  sfft_plan_destroy(p);
  cudaGetLastError();   // a failed candidate (e.g. out of memory) must not poison later calls
  return best;
}

}  // namespace

sfft_status_t autotune_tiles(const sfft_desc_t& d, cudaStream_t s, int d_batch_max, int* d_batch, int* rows_per_cta,
                             int* lag_parts, double* ms_per_ccd) {
  int dev = 0;
  cudaGetDevice(&dev);
  const std::string key = tune_key(d, dev);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache_file();
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *d_batch = it->second.d_batch;
      *rows_per_cta = it->second.rows_per_cta;
      *lag_parts = it->second.lag_parts;
      if (ms_per_ccd) *ms_per_ccd = it->second.ms;
      return SFFT_OK;
    }
  }
  std::vector<int> dbs = {d_batch_max};
  if (d_batch_max > 1) dbs.push_back((d_batch_max + 1) / 2);
  if (d.d_batch > 0) dbs = {d.d_batch};
  std::vector<int> rows;
  for (int r : {256, 512, 1024, 2048})
    if (r <= d.H) rows.push_back(r);
  if (rows.empty()) rows.push_back(d.H);
  if (d.rows_per_cta > 0) rows = {d.rows_per_cta};
  std::vector<int> parts = {2, 3};
  if (d.prec == SFFT_PREC_FP64) parts = {2};
  if (d.lag_parts > 0) parts = {d.lag_parts};
  Tuned best{0, 0, 0, -1.0};
  for (int db : dbs)
    for (int r : rows)
      for (int np : parts) {
        const double t = time_candidate(d, s, db, r, np);
        if (t > 0 && (best.ms < 0 || t < best.ms)) best = {db, r, np, t};
      }
  if (best.ms < 0) return SFFT_ERR_CUDA;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    store(key, best);
  }
  *d_batch = best.d_batch;
  *rows_per_cta = best.rows_per_cta;
  *lag_parts = best.lag_parts;
  if (ms_per_ccd) *ms_per_ccd = best.ms;
  return SFFT_OK;
}

}  // namespace sfft
