// noalloc.cu -- ct_apply_qt_noalloc: Q^T B with no device allocation.
//
// ct_apply_qt keeps the row-split partial products of V^T B in a workspace it
// allocates on the stream.  Some callers cannot have a library allocate
// device memory: an application whose framework has already reserved all of
// HBM for its own caching allocator (a library cudaMalloc then fails), or a
// latency-critical loop in which an allocation's implicit synchronisation is
// not acceptable.  This variant takes its workspace from a fixed array in the
// library's static device memory instead.
#include <mutex>

#include "internal.cuh"

namespace ctqr {
namespace {

// Limits of the static workspace: up to kMaxK right-hand sides per call and
// at most kMaxSplits row splits of V^T B (partials kMaxSplits x 64 x k, plus
// the 64 x k block W' = T^T V^T B), in doubles: 266,304 = 2.03 MiB.
constexpr int64_t kMaxK = 64;
constexpr int kMaxSplits = 64;
constexpr size_t kScratchElems = (size_t)(kMaxSplits + 1) * 64 * kMaxK + 64;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_apply_scratch[kScratchElems];

std::mutex g_mu;
// Device address of the array, per device (as many devices as device_info
// serves).  The address belongs to the device's primary context: after
// cudaDeviceReset the module is loaded again and this cached address is
// stale, so a process that resets a device must not call this entry point
// on it afterwards.
constexpr int kMaxDevices = 16;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (the host-side symbol is only a stand-in for it).
ct_status scratch_address(double** out) {
  int dev = 0;
  CT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return CT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_scratch);
    if (e != cudaSuccess || !p) {
      note_cuda_error(e, "cudaGetSymbolAddress(g_apply_scratch)", __FILE__, __LINE__);
      return CT_ERR_CUDA;
    }
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return CT_OK;
}

}  // namespace
}  // namespace ctqr

using namespace ctqr;

extern "C" ct_status ct_apply_qt_noalloc(const ct_factor* f, double* B, int64_t ldb, int64_t k, void* stream) {
  if (!f || k < 0) return CT_ERR_INVALID;
  if (k > kMaxK) return CT_ERR_INVALID;  // beyond the static workspace
  if (f->F_host) return CT_ERR_UNSUPPORTED;  // streaming a host factor allocates buffers
  if (k == 0) return CT_OK;
  if (!B || ((uintptr_t)B & 15u) || ldb < f->m) return CT_ERR_INVALID;
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  double* work = nullptr;
  if ((st = scratch_address(&work)) != CT_OK) return st;
  return apply_qt_all(f, B, true, ldb, k, false, work, kScratchElems, di.sms, (cudaStream_t)stream, kMaxSplits);
}
