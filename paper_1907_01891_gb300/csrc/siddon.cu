// siddon.cu -- dense system matrix A of Eq. (sistema): a_ij = length of ray i
// inside pixel j (Sec. II-A; the paper does not say how A is built, so this
// follows Siddon's ray traversal).  Compiled with -fmad=false so that every
// crossing parameter is the plain rounded sequence (line - p)/d.
//
// Work split: the m x n block is first zero-filled by a bandwidth-bound kernel
// (16-byte stores, grid a multiple of the SM count); then one thread per ray
// walks the grid lines it crosses, in order of the ray parameter t, and
// scatters the nonzero lengths (at most nx+ny per ray).  A ray only ever
// touches its own row, so the scatter needs no atomics.
#include <math.h>

#include "internal.cuh"

namespace ctqr {
namespace {

struct Geo {
  int beam, nx, ny, n_views, n_bins, angle_rule;
  double pixel, angle0, angle_span, src_iso, det_span, x0, y0;
};

// Angle of view v; angle_rule 1 adds the per-quarter shifts of Eq. (angulos)
// (0, +0.5, -0.25, -0.5 degrees; view i = v + 1 is in quarter q when
// q * n_views / 4 < i <= (q + 1) * n_views / 4).
__device__ __forceinline__ double view_angle(const Geo& g, int v) {
  double ang = g.angle0 + (double)v * g.angle_span / (double)g.n_views;
  if (g.angle_rule == 1) {
    const double i = (double)(v + 1), q4 = (double)g.n_views / 4.0;
    const double shift = i <= q4 ? 0.0 : (i <= 2.0 * q4 ? 0.5 : (i <= 3.0 * q4 ? -0.25 : -0.5));
    ang += shift * 3.14159265358979323846 / 180.0;
  }
  return ang;
}

__device__ __forceinline__ void ray_of(const Geo& g, int64_t ray, double& px, double& py,
                                       double& dx, double& dy) {
  const int v = (int)(ray / g.n_bins), b = (int)(ray % g.n_bins);
  const double ang = view_angle(g, v);
  const double c = (double)b - 0.5 * (double)(g.n_bins - 1);
  if (g.beam == 0) {
    const double s = c * (g.det_span / (double)g.n_bins);
    dx = cos(ang);
    dy = sin(ang);
    px = -s * dy;
    py = s * dx;
  } else {
    const double gam = g.n_bins > 1 ? c * (g.det_span / (double)(g.n_bins - 1)) : 0.0;
    px = g.src_iso * cos(ang);
    py = g.src_iso * sin(ang);
    dx = -cos(ang + gam);
    dy = -sin(ang + gam);
  }
}

// Grid line k along one axis: lo + k*pixel.
__device__ __forceinline__ double line(double lo, int k, double pixel) { return lo + (double)k * pixel; }

// Intersect [t0, t1] with {t : lo <= p + t d < hi} (half-open cell).
__device__ __forceinline__ void clip(double p, double d, double lo, double hi, double& t0, double& t1) {
  if (d == 0.0) {
    if (!(p >= lo && p < hi)) { t0 = 1.0; t1 = 0.0; }
    return;
  }
  const double ta = (lo - p) / d, tb = (hi - p) / d;
  const double tmin = ta < tb ? ta : tb, tmax = ta < tb ? tb : ta;
  if (tmin > t0) t0 = tmin;
  if (tmax < t1) t1 = tmax;
}

// Cell index k with line(k) <= x < line(k+1), clamped to [0, cells-1].
__device__ __forceinline__ int cell_of(double x, double lo, double pixel, int cells) {
  int k = (int)floor((x - lo) / pixel);
  k = k < 0 ? 0 : (k > cells - 1 ? cells - 1 : k);
  if (k > 0 && x < line(lo, k, pixel)) --k;
  if (k < cells - 1 && x >= line(lo, k + 1, pixel)) ++k;
  return k;
}

// Walk ray `ray` through the grid; emit(pixel, length) for every segment of
// positive length, in order of the ray parameter.  Returns the segment count.
template <typename Emit>
__device__ __forceinline__ int traverse(const Geo& g, int64_t ray, Emit emit) {
  double px, py, dx, dy;
  ray_of(g, ray, px, py, dx, dy);
  double t0 = -INFINITY, t1 = INFINITY;
  clip(px, dx, g.x0, line(g.x0, g.nx, g.pixel), t0, t1);
  clip(py, dy, g.y0, line(g.y0, g.ny, g.pixel), t0, t1);
  if (!(t1 > t0)) return 0;  // the ray misses the image

  // Next grid line to cross along x (index ix, stepping sx) and y.
  const int sx = dx > 0.0 ? 1 : -1, sy = dy > 0.0 ? 1 : -1;
  int ix = -1, iy = -1;
  if (dx != 0.0) {
    ix = (int)floor((px + t0 * dx - g.x0) / g.pixel) + (sx > 0 ? 0 : 1);
    ix = ix < 0 ? 0 : (ix > g.nx ? g.nx : ix);
    while (ix >= 0 && ix <= g.nx && (line(g.x0, ix, g.pixel) - px) / dx <= t0) ix += sx;
  }
  if (dy != 0.0) {
    iy = (int)floor((py + t0 * dy - g.y0) / g.pixel) + (sy > 0 ? 0 : 1);
    iy = iy < 0 ? 0 : (iy > g.ny ? g.ny : iy);
    while (iy >= 0 && iy <= g.ny && (line(g.y0, iy, g.pixel) - py) / dy <= t0) iy += sy;
  }
  double tcur = t0;
  int count = 0;
  const int max_steps = g.nx + g.ny + 4;
  for (int step = 0; step < max_steps && tcur < t1; ++step) {
    const double tx = (dx != 0.0 && ix >= 0 && ix <= g.nx) ? (line(g.x0, ix, g.pixel) - px) / dx : INFINITY;
    const double ty = (dy != 0.0 && iy >= 0 && iy <= g.ny) ? (line(g.y0, iy, g.pixel) - py) / dy : INFINITY;
    double tn = tx < ty ? tx : ty;
    if (t1 < tn) tn = t1;
    if (tn > tcur) {
      const double tm = 0.5 * (tcur + tn);
      const int cx = cell_of(px + tm * dx, g.x0, g.pixel, g.nx);
      const int cy = cell_of(py + tm * dy, g.y0, g.pixel, g.ny);
      emit(cy * g.nx + cx, tn - tcur);
      ++count;
    }
    if (tx <= tn) ix += sx;
    if (ty <= tn) iy += sy;
    tcur = tn;
  }
  return count;
}

template <typename S>
__global__ void __launch_bounds__(128) k_siddon(Geo g, S* __restrict__ A, int64_t lda) {
  const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rays = (int64_t)g.n_views * g.n_bins;
  if (ray >= rays) return;
  traverse(g, ray, [&](int j, double len) {
    S* dst = A + ray + (int64_t)j * lda;
    *dst = (S)((double)*dst + len);
  });
}

// Sparse form, pass 1: segments per ray.
__global__ void __launch_bounds__(128) k_ray_nnz(Geo g, int* __restrict__ nnz) {
  const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rays = (int64_t)g.n_views * g.n_bins;
  if (ray >= rays) return;
  nnz[ray] = traverse(g, ray, [](int, double) {});
}

// Sparse form, pass 2: CSR entries of every ray (same segments as k_siddon).
__global__ void __launch_bounds__(128) k_ray_fill(Geo g, const int64_t* __restrict__ row_ptr,
                                                  int* __restrict__ col, double* __restrict__ val) {
  const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rays = (int64_t)g.n_views * g.n_bins;
  if (ray >= rays) return;
  int64_t pos = row_ptr[ray];
  const int64_t end = row_ptr[ray + 1];
  traverse(g, ray, [&](int j, double len) {
    if (pos < end) {
      col[pos] = j;
      val[pos] = len;
      ++pos;
    }
  });
}

template <typename S>
__global__ void k_lambda_rows(S* __restrict__ A, int64_t lda, int64_t row0, int64_t n, double lambda) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) A[row0 + j + j * lda] = (S)lambda;
}

// Joseph's projector (the paper simulates its sinograms with it, Sec. III):
// one thread per (ray, image).  A ray with |dy| >= |dx| is sampled at every
// pixel row's centre line, where it falls between two pixel centres of that
// row; their values are interpolated linearly (a pixel outside the image
// counts as zero) and weighted by the step p / |dy|; otherwise the same with
// columns.  B[ray + c ldb] = the ray's sum for image c.
__global__ void __launch_bounds__(128) k_joseph(Geo g, const double* __restrict__ X, int64_t ldx, int64_t k,
                                                double* __restrict__ B, int64_t ldb) {
  const int64_t ray = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rays = (int64_t)g.n_views * g.n_bins;
  if (ray >= rays) return;
  double px, py, dx, dy;
  ray_of(g, ray, px, py, dx, dy);
  const bool by_rows = fabs(dy) >= fabs(dx);
  const int lines = by_rows ? g.ny : g.nx, cells = by_rows ? g.nx : g.ny;
  const double step = by_rows ? g.pixel / fabs(dy) : g.pixel / fabs(dx);
  for (int64_t c = blockIdx.y; c < k; c += gridDim.y) {
    const double* x = X + c * ldx;
    double acc = 0.0;
    for (int q = 0; q < lines; ++q) {
      double u;
      if (by_rows) {
        const double yc = g.y0 + ((double)q + 0.5) * g.pixel;
        const double t = (yc - py) / dy;
        u = (px + t * dx - g.x0) / g.pixel - 0.5;
      } else {
        const double xc = g.x0 + ((double)q + 0.5) * g.pixel;
        const double t = (xc - px) / dx;
        u = (py + t * dy - g.y0) / g.pixel - 0.5;
      }
      const double fl = floor(u), f = u - fl;
      const int64_t i0 = (int64_t)fl;
      double v = 0.0;
      if (i0 >= 0 && i0 < cells) v += (1.0 - f) * x[by_rows ? (int64_t)q * g.nx + i0 : i0 * g.nx + q];
      if (i0 + 1 >= 0 && i0 + 1 < cells) v += f * x[by_rows ? (int64_t)q * g.nx + i0 + 1 : (i0 + 1) * g.nx + q];
      acc += v;
    }
    B[ray + c * ldb] = step * acc;
  }
}

Geo make_geo(const ct_geometry* gg) {
  Geo g;
  g.beam = gg->beam; g.nx = gg->nx; g.ny = gg->ny; g.n_views = gg->n_views; g.n_bins = gg->n_bins;
  g.pixel = gg->pixel; g.angle0 = gg->angle0; g.angle_span = gg->angle_span;
  g.src_iso = gg->src_iso; g.det_span = gg->det_span; g.angle_rule = gg->angle_rule;
  g.x0 = -0.5 * (double)g.nx * g.pixel;
  g.y0 = -0.5 * (double)g.ny * g.pixel;
  return g;
}

}  // namespace

ct_status launch_ray_nnz(const ct_geometry* gg, int* nnz, cudaStream_t s) {
  const Geo g = make_geo(gg);
  const int64_t rays = (int64_t)g.n_views * g.n_bins;
  LaunchScope ls(K_SIDDON, s, 0.0, 4.0 * rays);
  k_ray_nnz<<<(unsigned)((rays + 127) / 128), 128, 0, s>>>(g, nnz);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status launch_ray_fill(const ct_geometry* gg, const int64_t* row_ptr, int* col, double* val, cudaStream_t s) {
  const Geo g = make_geo(gg);
  const int64_t rays = (int64_t)g.n_views * g.n_bins;
  LaunchScope ls(K_SIDDON, s, 0.0, 12.0 * rays * (g.nx + g.ny));
  k_ray_fill<<<(unsigned)((rays + 127) / 128), 128, 0, s>>>(g, row_ptr, col, val);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status launch_zero_matrix(void* A, size_t elem, int64_t lda, int64_t rows, int64_t cols,
                             cudaStream_t s);

ct_status launch_joseph(const ct_geometry* gg, const double* X, int64_t ldx, int64_t k, double* B, int64_t ldb,
                        cudaStream_t s) {
  const Geo g = make_geo(gg);
  const int64_t rays = (int64_t)g.n_views * g.n_bins;
  const unsigned gy = (unsigned)(k < 256 ? k : 256);
  LaunchScope ls(K_SIDDON, s, 3.0 * rays * (g.nx > g.ny ? g.nx : g.ny) * k, 16.0 * rays * (g.nx + g.ny) * k);
  k_joseph<<<dim3((unsigned)((rays + 127) / 128), gy), 128, 0, s>>>(g, X, ldx, k, B, ldb);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status launch_build_system(const ct_geometry* gg, ct_dtype dtype, double lambda, void* A,
                              int64_t lda, int64_t m, int64_t n, cudaStream_t s) {
  const Geo g = make_geo(gg);
  const size_t elem = dtype == CT_F64 ? 8 : 4;
  ct_status st = launch_zero_matrix(A, elem, lda, m, n, s);
  if (st != CT_OK) return st;
  const int64_t rays = (int64_t)g.n_views * g.n_bins;
  const unsigned blocks = (unsigned)((rays + 127) / 128);
  {
    LaunchScope ls(K_SIDDON, s, 0.0, (double)rays * (g.nx + g.ny) * elem);
    if (dtype == CT_F64) k_siddon<double><<<blocks, 128, 0, s>>>(g, (double*)A, lda);
    else k_siddon<float><<<blocks, 128, 0, s>>>(g, (float*)A, lda);
  }
  CT_LAUNCH_CHECK();
  if (lambda > 0.0) {
    LaunchScope ls(K_SIDDON, s, 0.0, (double)n * elem);
    if (dtype == CT_F64)
      k_lambda_rows<double><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((double*)A, lda, rays, n, lambda);
    else
      k_lambda_rows<float><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((float*)A, lda, rays, n, lambda);
    CT_LAUNCH_CHECK();
  }
  return CT_OK;
}

}  // namespace ctqr
