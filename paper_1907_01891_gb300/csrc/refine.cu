// refine.cu -- column-wise reductions and updates of the FP64 iterative
// refinement: X += D with per-column ||D_c||^2 and ||X_c||^2, and per-column
// squared norms.  One CTA per column; sums in a fixed order (deterministic).
#include "internal.cuh"

namespace ctqr {
namespace {

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(256) k_col_dots(const double* __restrict__ X, int64_t ldx,
                                                  const double* __restrict__ Y, int64_t ldy, int64_t rows,
                                                  double* __restrict__ out) {
  __shared__ double sh[8];
  const int64_t c = blockIdx.x;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) s += X[r + c * ldx] * Y[r + c * ldy];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[c] = s;
}

__global__ void __launch_bounds__(256) k_col_norms2(const double* __restrict__ X, int64_t ldx,
                                                    int64_t rows, double* __restrict__ out) {
  __shared__ double sh[8];
  const int64_t c = blockIdx.x;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
    const double v = X[r + c * ldx];
    s += v * v;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[c] = s;
}

template <typename TD>
__global__ void __launch_bounds__(256) k_add(const TD* __restrict__ D, int64_t ldd,
                                                 double* __restrict__ X, int64_t ldx, int64_t rows,
                                                 double* __restrict__ dn2, double* __restrict__ xn2) {
  __shared__ double sh[8];
  const int64_t c = blockIdx.x;
  double sd = 0.0, sx = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += blockDim.x) {
    const double d = (double)D[r + c * ldd];
    const double x = X[r + c * ldx] + d;
    X[r + c * ldx] = x;
    sd += d * d;
    sx += x * x;
  }
  sd = block_sum(sd, sh);
  if (threadIdx.x == 0) dn2[c] = sd;
  sx = block_sum(sx, sh);
  if (threadIdx.x == 0) xn2[c] = sx;
}

__global__ void __launch_bounds__(256) k_colwise(int mode, double sign, const double* __restrict__ a,
                                                 const double* __restrict__ X, int64_t ldx,
                                                 double* __restrict__ Y, int64_t ldy, int64_t rows) {
  const int64_t c = blockIdx.y;
  const double ac = a ? a[c] : 1.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (mode == 0) Y[r + c * ldy] += sign * ac * X[r + c * ldx];
    else Y[r + c * ldy] = X[r + c * ldx] + ac * Y[r + c * ldy];
  }
}

}  // namespace

ct_status launch_colwise(int mode, double sign, const double* a, const double* X, int64_t ldx,
                         double* Y, int64_t ldy, int64_t rows, int64_t k, cudaStream_t s) {
  if (rows <= 0 || k <= 0) return CT_OK;
  LaunchScope ls(K_AXPY, s, 2.0 * rows * k, 24.0 * rows * k);
  const unsigned gx = (unsigned)((rows + 255) / 256 < 128 ? (rows + 255) / 256 : 128);
  k_colwise<<<dim3(gx, (unsigned)k), 256, 0, s>>>(mode, sign, a, X, ldx, Y, ldy, rows);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status launch_col_dots(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t rows,
                          int64_t k, double* out, cudaStream_t s) {
  if (k <= 0) return CT_OK;
  LaunchScope ls(K_NORMS, s, 2.0 * rows * k, 16.0 * rows * k);
  k_col_dots<<<(unsigned)k, 256, 0, s>>>(X, ldx, Y, ldy, rows, out);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status launch_col_norms2(const double* X, int64_t ldx, int64_t rows, int64_t k, double* out,
                            cudaStream_t s) {
  if (k <= 0) return CT_OK;
  LaunchScope ls(K_NORMS, s, 2.0 * rows * k, 8.0 * rows * k);
  k_col_norms2<<<(unsigned)k, 256, 0, s>>>(X, ldx, rows, out);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status launch_add_f32_to_f64(const float* D, int64_t ldd, double* X, int64_t ldx, int64_t rows,
                                int64_t k, double* dnorm2, double* xnorm2, cudaStream_t s) {
  if (k <= 0) return CT_OK;
  LaunchScope ls(K_ADD, s, 4.0 * rows * k, 20.0 * rows * k);
  k_add<float><<<(unsigned)k, 256, 0, s>>>(D, ldd, X, ldx, rows, dnorm2, xnorm2);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status launch_add_f64_to_f64(const double* D, int64_t ldd, double* X, int64_t ldx, int64_t rows,
                                int64_t k, double* dnorm2, double* xnorm2, cudaStream_t s) {
  if (k <= 0) return CT_OK;
  LaunchScope ls(K_ADD, s, 4.0 * rows * k, 24.0 * rows * k);
  k_add<double><<<(unsigned)k, 256, 0, s>>>(D, ldd, X, ldx, rows, dnorm2, xnorm2);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

}  // namespace ctqr
