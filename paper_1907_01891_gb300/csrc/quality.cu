// quality.cu -- image quality of reconstructed slices (Sec. II-D): MSE
// (Eq. MSE), PSNR with the reference image's maximum (Eq. psnr) and SSIM
// (Eq. ssim); and the entry point of Joseph's projector (siddon.cu), the
// paper's sinogram simulator.
//
// SSIM's window and constants are not given in the paper; they are read as
// Wang et al.'s (2004): an 11 x 11 Gaussian window of sigma 1.5 normalised to
// sum 1, c1 = (0.01 L)^2, c2 = (0.03 L)^2 with L the reference's range
// (max - min), evaluated at every pixel whose window lies inside the image
// and averaged.  One CTA per slice; FP64 throughout.
#include <math.h>

#include "internal.cuh"

namespace ctqr {

ct_status launch_joseph(const ct_geometry* gg, const double* X, int64_t ldx, int64_t k, double* B, int64_t ldb,
                        cudaStream_t s);

namespace {

constexpr int kQT = 512;  // threads per slice
constexpr int kR = 5;     // window radius

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kQT / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  return sh[0];
}

__device__ __forceinline__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < kQT / 32 ? sh[threadIdx.x] : -INFINITY;
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) sh[0] = t;
  }
  __syncthreads();
  return sh[0];
}

// out[3c .. 3c+2] = MSE, PSNR (dB), SSIM of slice c of X against slice c of R.
__global__ void __launch_bounds__(kQT) k_quality(const double* __restrict__ X, int64_t ldx,
                                                 const double* __restrict__ R, int64_t ldr, int nx, int ny,
                                                 double* __restrict__ out) {
  __shared__ double sh[32];
  __shared__ double w[(2 * kR + 1) * (2 * kR + 1)];
  const int64_t c = blockIdx.x;
  const double* x = X + c * ldx;
  const double* r = R + c * ldr;
  const int64_t n = (int64_t)nx * ny;
  if (threadIdx.x < (2 * kR + 1) * (2 * kR + 1)) {
    const int a = threadIdx.x / (2 * kR + 1) - kR, b = threadIdx.x % (2 * kR + 1) - kR;
    w[threadIdx.x] = exp(-(double)(a * a + b * b) / (2.0 * 1.5 * 1.5));
  }
  double se = 0.0, mx = -INFINITY, mn = INFINITY;
  for (int64_t j = threadIdx.x; j < n; j += kQT) {
    const double d = x[j] - r[j];
    se += d * d;
    mx = fmax(mx, r[j]);
    mn = fmin(mn, r[j]);
  }
  const double sse = block_sum(se, sh);
  const double rmax = block_max(mx, sh);
  const double rmin = -block_max(-mn, sh);
  // window weights normalised to sum 1 (the same order of additions in every thread)
  double ws = 0.0;
  for (int q = 0; q < (2 * kR + 1) * (2 * kR + 1); ++q) ws += w[q];
  const double L = rmax - rmin, c1 = (0.01 * L) * (0.01 * L), c2 = (0.03 * L) * (0.03 * L);
  const int vx = nx - 2 * kR, vy = ny - 2 * kR;
  const int64_t valid = vx > 0 && vy > 0 ? (int64_t)vx * vy : 0;
  double ssum = 0.0;
  for (int64_t e = threadIdx.x; e < valid; e += kQT) {
    const int iy = (int)(e / vx) + kR, ix = (int)(e % vx) + kR;
    double mux = 0.0, muy = 0.0, sxx = 0.0, syy = 0.0, sxy = 0.0;
    for (int a = -kR; a <= kR; ++a) {
      const double* xr = x + (int64_t)(iy + a) * nx + ix;
      const double* rr = r + (int64_t)(iy + a) * nx + ix;
      for (int b = -kR; b <= kR; ++b) {
        const double wt = w[(a + kR) * (2 * kR + 1) + (b + kR)] / ws;
        const double xv = xr[b], rv = rr[b];
        mux += wt * xv;
        muy += wt * rv;
        sxx += wt * xv * xv;
        syy += wt * rv * rv;
        sxy += wt * xv * rv;
      }
    }
    const double varx = sxx - mux * mux, vary = syy - muy * muy, cov = sxy - mux * muy;
    ssum += ((2.0 * mux * muy + c1) * (2.0 * cov + c2)) / ((mux * mux + muy * muy + c1) * (varx + vary + c2));
  }
  const double stot = block_sum(ssum, sh);
  if (threadIdx.x == 0) {
    const double mse = sse / (double)n;
    out[3 * c] = mse;
    out[3 * c + 1] = 10.0 * log10(rmax * rmax / mse);
    out[3 * c + 2] = valid > 0 ? stot / (double)valid : NAN;
  }
}

}  // namespace
}  // namespace ctqr

using namespace ctqr;

extern "C" {

ct_status ct_project_joseph(const ct_geometry* g, const double* X, int64_t ldx, int64_t k, double* B, int64_t ldb,
                            void* stream) {
  int64_t m = 0, n = 0;
  ct_status st = ct_system_size(g, 0.0, &m, &n);
  if (st != CT_OK) return st;
  if (k < 0) return CT_ERR_INVALID;
  if (k == 0) return CT_OK;
  if (!X || !B || ldx < n || ldb < m) return CT_ERR_INVALID;
  return launch_joseph(g, X, ldx, k, B, ldb, (cudaStream_t)stream);
}

ct_status ct_image_quality(const double* X, int64_t ldx, const double* R, int64_t ldr, int nx, int ny, int64_t k,
                           double* out, void* stream) {
  if (nx < 1 || ny < 1 || k < 0) return CT_ERR_INVALID;
  if (k == 0) return CT_OK;
  const int64_t n = (int64_t)nx * ny;
  if (!X || !R || !out || ldx < n || ldr < n || k > 2147483647) return CT_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  LaunchScope ls(K_GATE, s, 10.0 * 121.0 * (double)n * k, 16.0 * (double)n * k);
  k_quality<<<(unsigned)k, kQT, 0, s>>>(X, ldx, R, ldr, nx, ny, out);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

}  // extern "C"
