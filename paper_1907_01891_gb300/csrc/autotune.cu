// autotune.cu -- measured choice of the batched tile-QR tile size.
//
// For a size class (GPU name, log2 of n, rows-per-column ratio in quarters)
// the tuner factors one synthetic system of that size with each candidate
// tile (32 and 64), keeps the faster, and caches the choice in a small JSON
// file ($CTQR_TUNE_CACHE, else $HOME/.cache/ctqr_tune.json) so later runs
// skip the measurement.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/stat.h>

#include <map>
#include <mutex>
#include <string>

#include "internal.cuh"

namespace ctqr {
namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_loaded = false;

std::string cache_path() {
  const char* p = getenv("CTQR_TUNE_CACHE");
  if (p && *p) return p;
  const char* h = getenv("HOME");
  return std::string(h ? h : "/tmp") + "/.cache/ctqr_tune.json";
}

// The file is a flat JSON object of "key": integer pairs.
void load_cache() {
  if (g_loaded) return;
  g_loaded = true;
  FILE* f = fopen(cache_path().c_str(), "r");
  if (!f) return;
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  fclose(f);
  size_t pos = 0;
  while ((pos = text.find('"', pos)) != std::string::npos) {
    const size_t end = text.find('"', pos + 1);
    if (end == std::string::npos) break;
    const std::string key = text.substr(pos + 1, end - pos - 1);
    const size_t colon = text.find(':', end);
    if (colon == std::string::npos) break;
    g_tune[key] = atoi(text.c_str() + colon + 1);
    pos = text.find_first_of(",}", colon);
    if (pos == std::string::npos) break;
  }
}

void save_cache() {
  const std::string path = cache_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);  // best effort
  FILE* f = fopen(path.c_str(), "w");
  if (!f) return;  // the cache is an optimisation only
  fprintf(f, "{");
  bool first = true;
  for (const auto& kv : g_tune) {
    fprintf(f, "%s\n  \"%s\": %d", first ? "" : ",", kv.first.c_str(), kv.second);
    first = false;
  }
  fprintf(f, "\n}\n");
  fclose(f);
}

__global__ void k_fill_synthetic(double* A, int64_t lda, int64_t m, int64_t n, uint64_t seed) {
  for (int64_t c = blockIdx.y; c < n; c += gridDim.y)
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
      uint64_t x = seed ^ (uint64_t)(r * 0x9E3779B97F4A7C15ull) ^ (uint64_t)(c * 0xC2B2AE3D27D4EB4Full);
      x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33;
      A[r + c * lda] = (double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5 + (r == c ? 4.0 : 0.0);
    }
}

}  // namespace

ct_status tuned_batch_tile(int64_t m, int64_t n, int sms, cudaStream_t s, int* tile) {
  cudaDeviceProp prop;
  int dev = 0;
  CT_CUDA_TRY(cudaGetDevice(&dev));
  CT_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  char key[256];
  const int ln = (int)floor(log2((double)(n > 1 ? n : 1)) + 0.5);
  const int ratio = (int)floor(4.0 * (double)m / (double)(n > 0 ? n : 1) + 0.5);
  snprintf(key, sizeof(key), "tile_qr/%s/log2n=%d/m_over_n_x4=%d", prop.name, ln, ratio);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_cache();
    auto it = g_tune.find(key);
    if (it != g_tune.end() && (it->second == 32 || it->second == 64)) {
      *tile = it->second;
      return CT_OK;
    }
  }
  // Measure: one synthetic m x n system (factor only) per candidate.
  const int64_t lda = m;
  double* A = nullptr;
  int* status = nullptr;
  CT_CUDA_TRY(cudaMallocAsync((void**)&A, (size_t)lda * n * sizeof(double) + 16, s));
  if (cudaMallocAsync((void**)&status, sizeof(int), s) != cudaSuccess) {
    cudaFreeAsync(A, s);
    return CT_ERR_NOMEM;
  }
  double best_ms = INFINITY;
  int best = 64;
  ct_status st = CT_OK;
  for (int cand : {32, 64}) {
    dim3 grid((unsigned)((m + 255) / 256 < 64 ? (m + 255) / 256 : 64), (unsigned)(n < 65535 ? n : 65535));
    k_fill_synthetic<<<grid, 256, 0, s>>>(A, lda, m, n, 12345);
    cudaMemsetAsync(status, 0, sizeof(int), s);
    ct_batch_system sys = {m, n, A, lda, nullptr, m, 0};
    double ms = 0.0;
    st = run_batch(1, &sys, cand, sms, status, s, &ms);
    if (st != CT_OK) break;
    if (ms < best_ms) { best_ms = ms; best = cand; }
  }
  cudaFreeAsync(A, s);
  cudaFreeAsync(status, s);
  if (st != CT_OK) return st;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best;
  save_cache();
  *tile = best;
  return CT_OK;
}

}  // namespace ctqr
