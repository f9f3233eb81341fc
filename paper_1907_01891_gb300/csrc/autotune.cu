// autotune.cu -- measured choices of the factorizations' block widths.
//
// Batched tile QR: for a size class (GPU name, log2 of n, rows-per-column
// ratio in quarters) the tuner factors one synthetic system of that size with
// each candidate tile (32 and 64) and keeps the faster.
// Tensor-core factorization: for a size class (GPU name, log2 of m and n,
// and the product arithmetic: 3xTF32, plain TF32 or the FP16 split) it
// factors a synthetic m x min(n, 2048) FP32 matrix with each panel width
// (16, 32) and, for TF32, each outer-block width (128, 256) and keeps the
// fastest; FP16-split factors keep 256-column outer blocks.
// Choices are cached in a small JSON file ($CTQR_TUNE_CACHE, else
// $HOME/.cache/ctqr_tune.json) so later runs skip the measurement.
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

__global__ void k_fill_synthetic_f32(float* A, int64_t lda, int64_t m, int64_t n, uint64_t seed) {
  for (int64_t c = blockIdx.y; c < n; c += gridDim.y)
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x) {
      uint64_t x = seed ^ (uint64_t)(r * 0x9E3779B97F4A7C15ull) ^ (uint64_t)(c * 0xC2B2AE3D27D4EB4Full);
      x ^= x >> 33; x *= 0xff51afd7ed558ccdull; x ^= x >> 33;
      A[r + c * lda] = (float)((double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    }
}

}  // namespace

ct_status tuned_factor_widths(int64_t m, int64_t n, int passes, ct_prec prec, cudaStream_t s, int* nb, int* outer) {
  *nb = 32;
  *outer = 256;
  const bool f16 = prec == CT_PREC_F16X3;
  const char* off = getenv("CTQR_NO_TUNE");
  if ((off && *off == '1') || n <= 128) return CT_OK;
  cudaDeviceProp prop;
  int dev = 0;
  CT_CUDA_TRY(cudaGetDevice(&dev));
  CT_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
  char key[256];
  const int lm = (int)floor(log2((double)m) + 0.5), ln = (int)floor(log2((double)n) + 0.5);
  if (f16)
    snprintf(key, sizeof(key), "factor_f16x3/%s/log2m=%d/log2n=%d", prop.name, lm, ln);
  else
    snprintf(key, sizeof(key), "factor_tf32/%s/passes=%d/log2m=%d/log2n=%d", prop.name, passes, lm, ln);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_cache();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      const int v = it->second, b = v / 1000, o = v % 1000;
      if ((b == 16 || b == 32) && (o == 128 || o == 256)) {
        *nb = b;
        *outer = o;
        return CT_OK;
      }
    }
  }
  // Measure on a synthetic m x nt FP32 matrix (the first columns of a system
  // of this shape: the panels' and updates' balance at full height).
  const int64_t nt = n < 2048 ? n : 2048, lda = (m + 3) / 4 * 4;
  float* A = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CT_CUDA_TRY(cudaMallocAsync((void**)&A, (size_t)lda * nt * sizeof(float) + 16, s));
  struct Free {
    float* a;
    cudaEvent_t* e0;
    cudaEvent_t* e1;
    cudaStream_t s;
    ~Free() {
      cudaFreeAsync(a, s);
      if (*e0) cudaEventDestroy(*e0);
      if (*e1) cudaEventDestroy(*e1);
    }
  } fr{A, &e0, &e1, s};
  CT_CUDA_TRY(cudaEventCreate(&e0));
  CT_CUDA_TRY(cudaEventCreate(&e1));
  const dim3 grid((unsigned)((m + 255) / 256 < 64 ? (m + 255) / 256 : 64), (unsigned)(nt < 65535 ? nt : 65535));
  k_fill_synthetic_f32<<<grid, 256, 0, s>>>(A, lda, m, nt, 777);
  CT_LAUNCH_CHECK();
  double best_ms = INFINITY;
  int best_nb = 32, best_outer = 256;
  for (int round = 0; round < 2; ++round) {  // round 0 loads the kernels, round 1 is timed
    for (int cand_nb : {16, 32}) {
      for (int cand_outer : {128, 256}) {
        if (round == 0 && !(cand_nb == 32 && cand_outer == 256)) continue;
        // FP16-split factors keep 256-column outer blocks: on the proxy's
        // 2048 columns 128 can look as fast, but on a wide matrix 256 halves
        // the passes over the trailing matrix, which bound these updates
        if (f16 && cand_outer != 256) continue;
        ct_qr_opts o = {cand_nb, 0, f16 ? 0 : passes, cand_outer};
        ct_factor* f = nullptr;
        CT_CUDA_TRY(cudaEventRecord(e0, s));
        ct_status st = ct_qr_factor(A, CT_F32, m, nt, lda, f16 ? CT_PREC_F16X3 : CT_PREC_TF32, &o, &f, s);
        if (st != CT_OK) return st;
        CT_CUDA_TRY(cudaEventRecord(e1, s));
        CT_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        CT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        const ct_status fs = ct_factor_status(f, s);
        ct_factor_destroy(f);
        if (fs != CT_OK && fs != CT_ERR_RANK) return fs;
        if (round == 1 && ms < best_ms) {
          best_ms = ms;
          best_nb = cand_nb;
          best_outer = cand_outer;
        }
      }
    }
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = best_nb * 1000 + best_outer;
  save_cache();
  *nb = best_nb;
  *outer = best_outer;
  return CT_OK;
}

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
    st = run_batch(1, &sys, cand, sms, status, s, false, &ms);
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
