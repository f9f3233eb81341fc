// util.cu -- bandwidth-bound helpers: zero fill and typed matrix copies.
#include <stdio.h>
#include <stdlib.h>

#include "internal.cuh"

namespace ctqr {

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  if (getenv("CTQR_VERBOSE"))
    fprintf(stderr, "ctqr: %s failed: %s (%s:%d)\n", what, cudaGetErrorString(e), file, line);
}

ct_status device_info(DeviceInfo* out) {
  static thread_local DeviceInfo cache[16];
  int dev = 0;
  CT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 16) return CT_ERR_UNSUPPORTED;
  if (cache[dev].device != dev) {
    DeviceInfo d;
    d.device = dev;
    CT_CUDA_TRY(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    CT_CUDA_TRY(cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cache[dev] = d;
  }
  *out = cache[dev];
  return CT_OK;
}

namespace {

// Zero `cols` columns of `rows` elements.  Contiguous case (ld == rows) uses
// 16-byte stores over the whole block; the grid is a multiple of the SM count.
__global__ void k_zero_flat(uint4* __restrict__ p, size_t n16, unsigned char* __restrict__ tail,
                            size_t ntail) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const uint4 z = make_uint4(0, 0, 0, 0);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) p[i] = z;
  if (blockIdx.x == 0)
    for (size_t i = threadIdx.x; i < ntail; i += blockDim.x) tail[i] = 0;
}

template <typename S>
__global__ void k_zero_cols(S* __restrict__ A, int64_t ld, int64_t rows, int64_t cols) {
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x)
      A[r + c * ld] = (S)0;
}

template <typename SS, typename DS>
__global__ void k_copy(const SS* __restrict__ src, int64_t lds, DS* __restrict__ dst, int64_t ldd,
                       int64_t rows, int64_t cols) {
  for (int64_t c = blockIdx.y; c < cols; c += gridDim.y)
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x)
      dst[r + c * ldd] = (DS)src[r + c * lds];
}

}  // namespace

ct_status launch_zero_matrix(void* A, size_t elem, int64_t lda, int64_t rows, int64_t cols,
                             cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return CT_OK;
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  if (lda == rows && ((uintptr_t)A % 16) == 0) {
    const size_t bytes = (size_t)rows * (size_t)cols * elem;
    const size_t n16 = bytes / 16;
    const unsigned grid = (unsigned)di.sms * 4;
    LaunchScope ls(K_ZERO, s, 0.0, (double)bytes);
    k_zero_flat<<<grid, 512, 0, s>>>((uint4*)A, n16, (unsigned char*)A + n16 * 16, bytes - n16 * 16);
  } else {
    dim3 grid((unsigned)((rows + 255) / 256 < 64 ? (rows + 255) / 256 : 64),
              (unsigned)(cols < 65535 ? cols : 65535));
    LaunchScope ls(K_ZERO, s, 0.0, (double)rows * cols * elem);
    if (elem == 8) k_zero_cols<double><<<grid, 256, 0, s>>>((double*)A, lda, rows, cols);
    else k_zero_cols<float><<<grid, 256, 0, s>>>((float*)A, lda, rows, cols);
  }
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status launch_copy_matrix(const void* src, ct_dtype st, int64_t lds, void* dst, ct_dtype dt,
                             int64_t ldd, int64_t rows, int64_t cols, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return CT_OK;
  dim3 grid((unsigned)((rows + 255) / 256 < 64 ? (rows + 255) / 256 : 64),
            (unsigned)(cols < 65535 ? cols : 65535));
  LaunchScope ls(K_COPY, s, 0.0,
                 (double)rows * cols * ((st == CT_F64 ? 8 : 4) + (dt == CT_F64 ? 8 : 4)));
  if (st == CT_F64 && dt == CT_F64)
    k_copy<double, double><<<grid, 256, 0, s>>>((const double*)src, lds, (double*)dst, ldd, rows, cols);
  else if (st == CT_F64 && dt == CT_F32)
    k_copy<double, float><<<grid, 256, 0, s>>>((const double*)src, lds, (float*)dst, ldd, rows, cols);
  else if (st == CT_F32 && dt == CT_F64)
    k_copy<float, double><<<grid, 256, 0, s>>>((const float*)src, lds, (double*)dst, ldd, rows, cols);
  else
    k_copy<float, float><<<grid, 256, 0, s>>>((const float*)src, lds, (float*)dst, ldd, rows, cols);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

}  // namespace ctqr
