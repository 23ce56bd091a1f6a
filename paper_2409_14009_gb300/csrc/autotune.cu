// autotune.cu -- the analysis-level autotuner of batched factorizations: which
// supernodes take the one-CTA kernel (small_max_cols / small_max_panel /
// small_max_rows), how much relaxed supernode merging to allow, and, per
// choice, the launch configuration (chol_autotune: level-by-level launches with
// or without graph replay, or the persistent cooperative kernel and its shape).
//
// Each candidate is timed on a deterministic sample of the batch (every k-th
// system), which keeps the search to seconds: every candidate needs its own
// symbolic analysis, and the analysis of the whole batch takes seconds by
// itself. The winner is kept in an optional text cache keyed by a hash of the
// pattern (systems, column pointers, row indices, permutation), the precision
// and update mode, and the device (name and SM count), so a later run on the
// same pattern skips the search.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "device.h"

namespace {

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct Cand {
  int32_t cols, panel, rows;
  double merge;
};

}  // namespace

extern "C" int chol_tune_batch(int32_t count, const int32_t* sys_ptr, const int64_t* colptr, const int32_t* rowind,
                               const int32_t* perm, const double* values, const chol_options* base,
                               int32_t sample_every, const char* cache_path, chol_options* best, double* best_ms,
                               int32_t* from_cache, void* stream) {
  NvtxRange nvtx_range("chol_tune_batch");
  if (count < 0) return -1;
  if (!sys_ptr) return -2;
  if (!colptr) return -3;
  if (!rowind && count > 0 && colptr[sys_ptr[count]] > 0) return -4;
  if (!values && count > 0 && colptr[sys_ptr[count]] > 0) return -6;
  if (sample_every < 1) return -8;
  if (!best) return -10;
  chol_options b0;
  if (base) b0 = *base; else chol_default_options(&b0);
  if (from_cache) *from_cache = 0;
  const int32_t n = count > 0 ? sys_ptr[count] : 0;
  const int64_t nnz = colptr[n];
  // cache key
  int dev = 0;
  cudaDeviceProp prop;
  CHOL_CUDA_TRY(cudaGetDevice(&dev));
  CHOL_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  uint64_t key = 1469598103934665603ull;
  key = fnv1a(key, &count, sizeof(count));
  key = fnv1a(key, sys_ptr, sizeof(int32_t) * (size_t)(count + 1));
  key = fnv1a(key, colptr, sizeof(int64_t) * (size_t)(n + 1));
  if (nnz > 0) key = fnv1a(key, rowind, sizeof(int32_t) * (size_t)nnz);
  if (perm) key = fnv1a(key, perm, sizeof(int32_t) * (size_t)n);
  key = fnv1a(key, &b0.precision, sizeof(b0.precision));
  key = fnv1a(key, &b0.update_mode, sizeof(b0.update_mode));
  key = fnv1a(key, prop.name, std::strlen(prop.name));
  key = fnv1a(key, &prop.multiProcessorCount, sizeof(int));
  char keystr[32];
  std::snprintf(keystr, sizeof(keystr), "%016llx", (unsigned long long)key);
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string k;
      chol_options o = b0;
      double ms = 0.0;
      if (ls >> k >> o.small_max_cols >> o.small_max_panel >> o.small_max_rows >> o.merge_growth >> o.persistent >>
              o.use_graph >> ms &&
          k == keystr) {
        *best = o;
        if (best_ms) *best_ms = ms;
        if (from_cache) *from_cache = 1;
        return CHOL_OK;
      }
    }
  }
  // the sample: every sample_every-th system, rebased into one block-diagonal matrix
  std::vector<int32_t> sptr{0};
  std::vector<int64_t> cp{0};
  std::vector<int32_t> ri, pm;
  std::vector<std::pair<int64_t, int64_t>> segs;   // value ranges of the sampled systems
  for (int32_t q = 0; q < count; q += sample_every) {
    const int32_t c0 = sys_ptr[q], c1 = sys_ptr[q + 1], base_col = sptr.back();
    for (int32_t j = c0; j < c1; ++j) {
      for (int64_t t = colptr[j]; t < colptr[j + 1]; ++t) ri.push_back(rowind[t] - c0 + base_col);
      cp.push_back((int64_t)ri.size());
      pm.push_back((perm ? perm[j] : j) - c0 + base_col);
    }
    segs.push_back({colptr[c0], colptr[c1]});
    sptr.push_back(base_col + (c1 - c0));
  }
  const int32_t scount = (int32_t)sptr.size() - 1;
  const int64_t snnz = (int64_t)ri.size();
  cudaStream_t st = (cudaStream_t)stream;
  double* svals = nullptr;
  CHOL_CUDA_TRY(cudaMalloc(&svals, sizeof(double) * (size_t)std::max<int64_t>(snnz, 1)));
  {
    int64_t off = 0;
    for (const auto& sg : segs) {
      const int64_t len = sg.second - sg.first;
      if (len > 0 && cudaMemcpyAsync(svals + off, values + sg.first, sizeof(double) * (size_t)len,
                                     cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
        cudaFree(svals);
        return CHOL_ECUDA;
      }
      off += len;
    }
  }
  const std::vector<Cand> cands = {{64, 4096, 128, 0.0},    {64, 4096, 128, 0.1},    {64, 4096, 128, 0.25},
                                   {128, 16384, 256, 0.0},  {128, 16384, 256, 0.1},  {128, 16384, 256, 0.25},
                                   {160, 24576, 512, 0.0},  {160, 24576, 512, 0.1},  {160, 24576, 512, 0.25}};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaFree(svals);
    return CHOL_ECUDA;
  }
  int rc = CHOL_OK;
  double bms = 1e300;
  chol_options bopt = b0;
  for (const Cand& c : cands) {
    chol_options o = b0;
    o.small_max_cols = c.cols;
    o.small_max_panel = c.panel;
    o.small_max_rows = c.rows;
    o.merge_growth = c.merge;
    o.persistent = 0;
    o.use_graph = 0;
    chol_handle* h = nullptr;
    rc = chol_analyze_batch(scount, sptr.data(), cp.data(), ri.data(), pm.data(), &o, &h);
    if (rc) break;
    rc = chol_autotune(h, svals, stream);   // launch configuration for this analysis; leaves h factored
    float tmin = 1e30f;
    for (int rep = 0; rep < 3 && rc == CHOL_OK; ++rep) {
      cudaEventRecord(e0, st);
      rc = chol_factor(h, svals, stream);
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      tmin = std::min(tmin, ms);
    }
    if (rc == CHOL_OK && tmin < bms) {
      bms = tmin;
      bopt = o;
      bopt.persistent = h->opt.persistent;
      bopt.use_graph = h->opt.use_graph;
    }
    chol_destroy(h);
    if (rc) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(svals);
  if (rc) return rc;
  *best = bopt;
  if (best_ms) *best_ms = bms;
  if (cache_path) {
    std::ofstream out(cache_path, std::ios::app);
    out << keystr << ' ' << bopt.small_max_cols << ' ' << bopt.small_max_panel << ' ' << bopt.small_max_rows << ' '
        << bopt.merge_growth << ' ' << bopt.persistent << ' ' << bopt.use_graph << ' ' << bms << '\n';
  }
  return CHOL_OK;
}
