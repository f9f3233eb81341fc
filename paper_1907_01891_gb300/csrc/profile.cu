// profile.cu -- launch accounting and optional CUDA-event timing per kernel
// class.  Every kernel launch of the library goes through a LaunchScope, which
// counts it and, when timing is enabled, records a start/stop event pair on
// the launching stream.  ct_profile_kernels() synchronises those events and
// reports launches, device time and the launch's algorithmic flops / bytes.
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace ctqr {
namespace {

struct Pending {
  cudaEvent_t a, b;
  int cls;
};

struct Profiler {
  std::mutex mu;
  bool timing = false;
  bool capturing = false;           // launches are being recorded into a graph
  uint64_t captured[K_COUNT] = {};  // launches recorded since begin_capture
  double captured_flops[K_COUNT] = {};
  uint64_t launches[K_COUNT] = {};
  uint64_t timed[K_COUNT] = {};
  double ms[K_COUNT] = {};
  double flops[K_COUNT] = {};
  double bytes[K_COUNT] = {};
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;

  cudaEvent_t get_event() {
    if (!free_events.empty()) {
      cudaEvent_t e = free_events.back();
      free_events.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
  void drain() {
    for (const Pending& p : pending) {
      float t = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
        ms[p.cls] += t;
        timed[p.cls] += 1;
      } else {
        cudaGetLastError();
      }
      free_events.push_back(p.a);
      free_events.push_back(p.b);
    }
    pending.clear();
  }
};

Profiler& prof() {
  static Profiler* p = new Profiler;  // never destroyed: events outlive static teardown
  return *p;
}

const char* kNames[K_COUNT] = {"zero_fill",   "system_matrix", "panel_qr",  "reflector_vtc",
                               "reflector_tw", "block_update",  "trsm_diag", "copy",
                               "rank_check",  "col_norms",     "col_add",   "gemm_tn",
                               "col_axpy",    "tc_gemm",       "spmm",      "tile_runtime",
                               "conv",        "gate",          "tc_update",
                               "qt_outer",    "inner_update",  "t_inverse"};

}  // namespace

LaunchScope::LaunchScope(int cls, cudaStream_t s, double flops, double bytes)
    : cls_(cls), s_(s), start_(nullptr) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  if (p.capturing) {  // recorded into a graph: counted when the graph is replayed
    p.captured[cls] += 1;
    p.captured_flops[cls] += flops;
    return;
  }
  p.launches[cls] += 1;
  p.flops[cls] += flops;
  p.bytes[cls] += bytes;
  if (p.timing) {
    start_ = p.get_event();
    if (start_) cudaEventRecord((cudaEvent_t)start_, s);
  }
}

LaunchScope::~LaunchScope() {
  if (!start_) return;
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  cudaEvent_t stop = p.get_event();
  if (!stop) return;
  cudaEventRecord(stop, s_);
  p.pending.push_back({(cudaEvent_t)start_, stop, cls_});
}

void profile_begin_capture() {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.capturing = true;
  for (int i = 0; i < K_COUNT; ++i) {
    p.captured[i] = 0;
    p.captured_flops[i] = 0.0;
  }
}

void profile_end_capture(GraphCounts* out) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.capturing = false;
  for (int i = 0; i < K_COUNT; ++i) {
    out->launches[i] = p.captured[i];
    out->flops[i] = p.captured_flops[i];
  }
}

void profile_note_replay(const GraphCounts& c) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  for (int i = 0; i < K_COUNT; ++i) {
    p.launches[i] += c.launches[i];
    p.flops[i] += c.flops[i];
  }
}

}  // namespace ctqr

using namespace ctqr;

extern "C" {

void ct_profile_enable(int on) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.timing = on != 0;
}

void ct_profile_reset(void) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.drain();
  for (int i = 0; i < K_COUNT; ++i) {
    p.launches[i] = p.timed[i] = 0;
    p.ms[i] = p.flops[i] = p.bytes[i] = 0.0;
  }
}

int ct_profile_kernels(ct_kernel_stats* out, int max_entries) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.drain();
  int n = 0;
  for (int i = 0; i < K_COUNT && n < max_entries; ++i) {
    if (!out) break;
    out[n].name = kNames[i];
    out[n].launches = p.launches[i];
    out[n].timed = p.timed[i];
    out[n].ms = p.ms[i];
    out[n].flops = p.flops[i];
    out[n].bytes = p.bytes[i];
    ++n;
  }
  return out ? n : K_COUNT;
}

uint64_t ct_kernel_launches(void) {
  Profiler& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  uint64_t s = 0;
  for (int i = 0; i < K_COUNT; ++i) s += p.launches[i];
  return s;
}

}  // extern "C"
