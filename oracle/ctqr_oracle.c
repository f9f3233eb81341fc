/*
 * ctqr_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the
 * QR-based CT reconstruction hot path.  TEST INFRASTRUCTURE ONLY: only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark load it.
 * It shares no code, header or constant with the CUDA library.
 *
 * What it computes (paper: Chillaron et al., "Computed tomography medical image
 * reconstruction on affordable equipment by using out-of-core techniques"):
 *   - the system matrix A of Eq. (sistema): a_ij = contribution of ray i to
 *     pixel j, read as the length of ray i inside pixel j (Sec. II-A);
 *   - the Householder QR factorization A = QR of Eq. (QR), reflectors stored
 *     below the diagonal and R on and above it, as the Compute_dense_QR task
 *     describes (Sec. II-C-3);
 *   - the implicit application of Q^T to the sinograms B (first sub-step of
 *     X = R^{-1}(Q^T B), Eq. (qr1), Sec. II-C-4);
 *   - backward substitution with the upper triangular R (second sub-step of
 *     Eq. (qr1), Sec. II-C-4);
 *   - a direct 3x3 convolution forward/backward pass used to check the
 *     surrogate network's kernels.
 * Everything is column-major (element (i,j) of a matrix with leading
 * dimension ld sits at [i + j*ld]) and computed in IEEE double precision.
 * Build with -ffp-contract=off so no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* ------------------------------------------------------------------------ */
/* Scanner geometry.  Rays are numbered ray = view * n_bins + bin.           */
/*  beam 0 (parallel): theta_v = angle0 + v*angle_span/n_views; bin offset   */
/*    s_b = (b - (n_bins-1)/2) * det_span/n_bins; the ray passes through     */
/*    s_b*(-sin th, cos th) with direction (cos th, sin th).                 */
/*  beam 1 (fan, equiangular): source angle beta_v as above, source at       */
/*    src_iso*(cos b, sin b); fan angle g_b = (b-(n_bins-1)/2)*det_span/     */
/*    (n_bins-1) (0 when n_bins == 1); direction (-cos(beta+g), -sin(beta+g)).*/
/* The image has nx*ny square pixels of side `pixel`, centred on the origin; */
/* pixel j = iy*nx + ix covers [x0+ix*p, x0+(ix+1)*p) x [y0+iy*p, ...).      */
/* angle_rule 1: the views of Eq. (angulos), read as the uniform angles      */
/* shifted per quarter of the views by 0, +0.5, -0.25 and -0.5 degrees       */
/* (the equation's +0.5, -0.75, -0.25 taken relative to the previous         */
/* quarter); view i (1-based) is in quarter q when q*v/4 < i <= (q+1)*v/4.   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int beam, nx, ny;
  double pixel;
  int n_views, n_bins;
  double angle0, angle_span, src_iso, det_span;
  int angle_rule;
} og_geometry;

/* Angle (radians) of view v (0-based). */
double oracle_view_angle(const og_geometry* g, int v) {
  double ang = g->angle0 + (double)v * g->angle_span / (double)g->n_views;
  if (g->angle_rule == 1) {
    const double pi = 3.14159265358979323846;
    const double i = (double)(v + 1), q4 = (double)g->n_views / 4.0;
    double shift_deg = 0.0;
    if (i <= q4) shift_deg = 0.0;
    else if (i <= 2.0 * q4) shift_deg = 0.5;
    else if (i <= 3.0 * q4) shift_deg = 0.5 - 0.75;
    else shift_deg = 0.5 - 0.75 - 0.25;
    ang += shift_deg * pi / 180.0;
  }
  return ang;
}

void oracle_ray(const og_geometry* g, int64_t ray, double* px, double* py,
                double* dx, double* dy) {
  int v = (int)(ray / g->n_bins), b = (int)(ray % g->n_bins);
  double ang = oracle_view_angle(g, v);
  double c = (double)b - 0.5 * (double)(g->n_bins - 1);
  if (g->beam == 0) {
    double s = c * (g->det_span / (double)g->n_bins);
    *dx = cos(ang);
    *dy = sin(ang);
    *px = -s * (*dy);
    *py = s * (*dx);
  } else {
    /* a one-bin fan is just its central ray */
    double gam = g->n_bins > 1 ? c * (g->det_span / (double)(g->n_bins - 1)) : 0.0;
    *px = g->src_iso * cos(ang);
    *py = g->src_iso * sin(ang);
    *dx = -cos(ang + gam);
    *dy = -sin(ang + gam);
  }
}

/* Parameter interval {t : lo <= p + t*d < hi} intersected into [*t0, *t1].
 * Half-open cells: a ray lying exactly on a line belongs to the cell above it. */
static void clip_slab(double p, double d, double lo, double hi, double* t0,
                      double* t1) {
  if (d == 0.0) {
    if (!(p >= lo && p < hi)) { *t0 = 1.0; *t1 = 0.0; }
    return;
  }
  double ta = (lo - p) / d, tb = (hi - p) / d;
  double tmin = ta < tb ? ta : tb, tmax = ta < tb ? tb : ta;
  if (tmin > *t0) *t0 = tmin;
  if (tmax < *t1) *t1 = tmax;
}

/* a_ij = length of ray i inside pixel j, straight from the definition: clip
 * the ray's line against every pixel square.  O(m*n) work. */
void oracle_system_matrix(const og_geometry* g, double* A, int64_t lda) {
  int64_t m = (int64_t)g->n_views * g->n_bins;
  int64_t n = (int64_t)g->nx * g->ny;
  double x0 = -0.5 * (double)g->nx * g->pixel;
  double y0 = -0.5 * (double)g->ny * g->pixel;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; i++) {
    double px, py, dx, dy;
    oracle_ray(g, i, &px, &py, &dx, &dy);
    for (int iy = 0; iy < g->ny; iy++) {
      for (int ix = 0; ix < g->nx; ix++) {
        double t0 = -INFINITY, t1 = INFINITY;
        clip_slab(px, dx, x0 + ix * g->pixel, x0 + (ix + 1) * g->pixel, &t0, &t1);
        clip_slab(py, dy, y0 + iy * g->pixel, y0 + (iy + 1) * g->pixel, &t0, &t1);
        A[IDX(i, (int64_t)iy * g->nx + ix, lda)] = t1 > t0 ? t1 - t0 : 0.0;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Joseph's projector (the paper simulates its sinograms with it, Sec. III;  */
/* Joseph, "An improved algorithm for reprojecting rays through pixel        */
/* images", 1982).  For a ray with unit direction (dx, dy): when             */
/* |dy| >= |dx| it crosses every pixel row; at row iy's centre line          */
/* y_c = y0 + (iy + 1/2) p it is at x(y_c), which lies between the centres    */
/* of columns i0 and i0 + 1 with u = (x - x0)/p - 1/2, i0 = floor(u),         */
/* f = u - i0; the row contributes p/|dy| * ((1 - f) X[iy, i0] + f X[iy, i0+1]), */
/* a pixel outside the image counting as zero.  Otherwise the same with the  */
/* roles of rows and columns exchanged (step p/|dx|).                        */
/* B[i, c] = sum over rows (or columns) for image c.                         */
/* ------------------------------------------------------------------------ */
void oracle_joseph(const og_geometry* g, const double* X, int64_t ldx, int64_t k, double* B, int64_t ldb) {
  int64_t m = (int64_t)g->n_views * g->n_bins;
  double p = g->pixel;
  double x0 = -0.5 * (double)g->nx * p;
  double y0 = -0.5 * (double)g->ny * p;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; i++) {
    double px, py, dx, dy;
    oracle_ray(g, i, &px, &py, &dx, &dy);
    int by_rows = fabs(dy) >= fabs(dx);
    int lines = by_rows ? g->ny : g->nx;
    int cells = by_rows ? g->nx : g->ny;
    double step = by_rows ? p / fabs(dy) : p / fabs(dx);
    for (int64_t c = 0; c < k; c++) {
      double acc = 0.0;
      for (int q = 0; q < lines; q++) {
        double u;
        if (by_rows) {
          double yc = y0 + ((double)q + 0.5) * p;
          double t = (yc - py) / dy;
          double x = px + t * dx;
          u = (x - x0) / p - 0.5;
        } else {
          double xc = x0 + ((double)q + 0.5) * p;
          double t = (xc - px) / dx;
          double y = py + t * dy;
          u = (y - y0) / p - 0.5;
        }
        double fl = floor(u);
        double f = u - fl;
        int64_t i0 = (int64_t)fl;
        double v = 0.0;
        if (i0 >= 0 && i0 < cells) {
          int64_t j = by_rows ? (int64_t)q * g->nx + i0 : i0 * g->nx + q;
          v += (1.0 - f) * X[IDX(j, c, ldx)];
        }
        if (i0 + 1 >= 0 && i0 + 1 < cells) {
          int64_t j = by_rows ? (int64_t)q * g->nx + (i0 + 1) : (i0 + 1) * g->nx + q;
          v += f * X[IDX(j, c, ldx)];
        }
        acc += v;
      }
      B[IDX(i, c, ldb)] = step * acc;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Image quality of Sec. II-D: MSE (Eq. MSE), PSNR with the reference's       */
/* maximum (Eq. psnr) and SSIM (Eq. ssim).  The paper leaves SSIM's window   */
/* and constants open; the reading (Wang et al. 2004): an 11 x 11 Gaussian   */
/* window of sigma 1.5 (weights normalised to sum 1), c1 = (0.01 L)^2,       */
/* c2 = (0.03 L)^2 with L = max - min of the reference, SSIM evaluated at    */
/* every pixel whose whole window lies in the image and averaged.            */
/* x, ref: one image each (pixel iy*nx + ix).  out[0] = MSE, out[1] = PSNR   */
/* (dB), out[2] = SSIM.                                                      */
/* ------------------------------------------------------------------------ */
void oracle_quality(const double* x, const double* ref, int nx, int ny, double* out) {
  int64_t n = (int64_t)nx * ny;
  double mse = 0.0, mx = -INFINITY, mn = INFINITY;
  for (int64_t j = 0; j < n; j++) {
    double d = x[j] - ref[j];
    mse += d * d;
    if (ref[j] > mx) mx = ref[j];
    if (ref[j] < mn) mn = ref[j];
  }
  mse /= (double)n;
  out[0] = mse;
  out[1] = 10.0 * log10(mx * mx / mse);
  const int R = 5;
  double w[11 * 11], ws = 0.0;
  for (int a = -R; a <= R; a++)
    for (int b = -R; b <= R; b++) {
      double e = exp(-(double)(a * a + b * b) / (2.0 * 1.5 * 1.5));
      w[(a + R) * 11 + (b + R)] = e;
      ws += e;
    }
  for (int q = 0; q < 121; q++) w[q] /= ws;
  double L = mx - mn;
  double c1 = (0.01 * L) * (0.01 * L), c2 = (0.03 * L) * (0.03 * L);
  double total = 0.0;
  int64_t count = 0;
  for (int iy = R; iy < ny - R; iy++) {
    for (int ix = R; ix < nx - R; ix++) {
      double mux = 0.0, muy = 0.0, sxx = 0.0, syy = 0.0, sxy = 0.0;
      for (int a = -R; a <= R; a++)
        for (int b = -R; b <= R; b++) {
          double wt = w[(a + R) * 11 + (b + R)];
          int64_t j = (int64_t)(iy + a) * nx + (ix + b);
          mux += wt * x[j];
          muy += wt * ref[j];
          sxx += wt * x[j] * x[j];
          syy += wt * ref[j] * ref[j];
          sxy += wt * x[j] * ref[j];
        }
      double vx = sxx - mux * mux, vy = syy - muy * muy, cxy = sxy - mux * muy;
      total += ((2.0 * mux * muy + c1) * (2.0 * cxy + c2)) /
               ((mux * mux + muy * muy + c1) * (vx + vy + c2));
      count++;
    }
  }
  out[2] = count > 0 ? total / (double)count : NAN;
}

/* ------------------------------------------------------------------------ */
/* Householder QR, unblocked (column by column).  For column j:              */
/*   alpha = A[j,j], sigma = sum_{i>j} A[i,j]^2.                             */
/*   sigma == 0: tau_j = 0, nothing changes (H_j = I).                       */
/*   else: mu = sqrt(alpha^2 + sigma), beta = -mu if alpha >= 0 else mu,     */
/*         tau_j = (beta - alpha)/beta, v = A[j:m,j]/(alpha - beta), v_0 = 1;*/
/*         A[j,j] = beta, A[j+1:m,j] = v[1:]; every later column c gets      */
/*         A[j:m,c] -= tau_j * (v^T A[j:m,c]) * v.                           */
/* H_j = I - tau_j v v^T, Q = H_0 H_1 ... H_{n-1}, A = QR.                    */
/* ------------------------------------------------------------------------ */
void oracle_qr(double* A, int64_t m, int64_t n, int64_t lda, double* tau) {
  int64_t kmax = m < n ? m : n;
  for (int64_t j = 0; j < kmax; j++) {
    double alpha = A[IDX(j, j, lda)];
    double sigma = 0.0;
    for (int64_t i = j + 1; i < m; i++) sigma += A[IDX(i, j, lda)] * A[IDX(i, j, lda)];
    if (sigma == 0.0) { tau[j] = 0.0; continue; }
    double mu = sqrt(alpha * alpha + sigma);
    double beta = alpha >= 0.0 ? -mu : mu;
    double t = (beta - alpha) / beta;
    for (int64_t i = j + 1; i < m; i++) A[IDX(i, j, lda)] /= (alpha - beta);
    A[IDX(j, j, lda)] = beta;
    tau[j] = t;
#pragma omp parallel for schedule(static)
    for (int64_t c = j + 1; c < n; c++) {
      double w = A[IDX(j, c, lda)];
      for (int64_t i = j + 1; i < m; i++) w += A[IDX(i, j, lda)] * A[IDX(i, c, lda)];
      w *= t;
      A[IDX(j, c, lda)] -= w;
      for (int64_t i = j + 1; i < m; i++) A[IDX(i, c, lda)] -= w * A[IDX(i, j, lda)];
    }
  }
}

/* B <- Q^T B = H_{n-1} ... H_1 H_0 B, reflectors taken from oracle_qr's output. */
void oracle_apply_qt(const double* F, int64_t m, int64_t n, int64_t lda,
                     const double* tau, double* B, int64_t ldb, int64_t k) {
  int64_t kmax = m < n ? m : n;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < k; c++) {
    for (int64_t j = 0; j < kmax; j++) {
      if (tau[j] == 0.0) continue;
      double w = B[IDX(j, c, ldb)];
      for (int64_t i = j + 1; i < m; i++) w += F[IDX(i, j, lda)] * B[IDX(i, c, ldb)];
      w *= tau[j];
      B[IDX(j, c, ldb)] -= w;
      for (int64_t i = j + 1; i < m; i++) B[IDX(i, c, ldb)] -= w * F[IDX(i, j, lda)];
    }
  }
}

/* B <- Q B = H_0 H_1 ... H_{n-1} B (used only to check Q in the tests). */
void oracle_apply_q(const double* F, int64_t m, int64_t n, int64_t lda,
                    const double* tau, double* B, int64_t ldb, int64_t k) {
  int64_t kmax = m < n ? m : n;
  for (int64_t c = 0; c < k; c++) {
    for (int64_t j = kmax - 1; j >= 0; j--) {
      if (tau[j] == 0.0) continue;
      double w = B[IDX(j, c, ldb)];
      for (int64_t i = j + 1; i < m; i++) w += F[IDX(i, j, lda)] * B[IDX(i, c, ldb)];
      w *= tau[j];
      B[IDX(j, c, ldb)] -= w;
      for (int64_t i = j + 1; i < m; i++) B[IDX(i, c, ldb)] -= w * F[IDX(i, j, lda)];
    }
  }
}

/* Solve R X = Y by backward substitution, X overwriting Y[0:n, 0:k].
 * Returns 0, or 4 if some |R_ii| <= max(m,n) * eps * max_i |R_ii|
 * (numerically rank deficient; X is then left untouched). */
int oracle_backsolve(const double* F, int64_t m, int64_t n, int64_t lda,
                     double* Y, int64_t ldy, int64_t k) {
  double rmax = 0.0;
  for (int64_t i = 0; i < n; i++) {
    double r = fabs(F[IDX(i, i, lda)]);
    if (r > rmax) rmax = r;
  }
  double thr = (double)(m > n ? m : n) * 2.220446049250313e-16 * rmax;
  for (int64_t i = 0; i < n; i++)
    if (!(fabs(F[IDX(i, i, lda)]) > thr)) return 4;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < k; c++) {
    for (int64_t i = n - 1; i >= 0; i--) {
      double s = Y[IDX(i, c, ldy)];
      for (int64_t l = i + 1; l < n; l++) s -= F[IDX(i, l, lda)] * Y[IDX(l, c, ldy)];
      Y[IDX(i, c, ldy)] = s / F[IDX(i, i, lda)];
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 3x3 convolution, stride 1, zero padding 1, NCHW, FP64.                    */
/*   y[b,o,h,w] = bias[o] + sum_{c,dh,dw} wt[o,c,dh,dw] x[b,c,h+dh-1,w+dw-1] */
/* and the gradients of sum(gy * y) w.r.t. x, wt and bias.                   */
/* ------------------------------------------------------------------------ */
void oracle_conv3x3_fwd(const double* x, const double* wt, const double* bias,
                        double* y, int B, int C, int O, int H, int W) {
  for (int b = 0; b < B; b++)
    for (int o = 0; o < O; o++)
      for (int h = 0; h < H; h++)
        for (int w = 0; w < W; w++) {
          double s = bias ? bias[o] : 0.0;
          for (int c = 0; c < C; c++)
            for (int dh = 0; dh < 3; dh++)
              for (int dw = 0; dw < 3; dw++) {
                int hh = h + dh - 1, ww = w + dw - 1;
                if (hh < 0 || hh >= H || ww < 0 || ww >= W) continue;
                s += wt[((size_t)(o * C + c) * 3 + dh) * 3 + dw] *
                     x[(((size_t)b * C + c) * H + hh) * W + ww];
              }
          y[(((size_t)b * O + o) * H + h) * W + w] = s;
        }
}

void oracle_conv3x3_bwd(const double* x, const double* wt, const double* gy,
                        double* gx, double* gw, double* gb, int B, int C, int O,
                        int H, int W) {
  memset(gx, 0, sizeof(double) * (size_t)B * C * H * W);
  memset(gw, 0, sizeof(double) * (size_t)O * C * 9);
  memset(gb, 0, sizeof(double) * (size_t)O);
  for (int b = 0; b < B; b++)
    for (int o = 0; o < O; o++)
      for (int h = 0; h < H; h++)
        for (int w = 0; w < W; w++) {
          double g = gy[(((size_t)b * O + o) * H + h) * W + w];
          gb[o] += g;
          for (int c = 0; c < C; c++)
            for (int dh = 0; dh < 3; dh++)
              for (int dw = 0; dw < 3; dw++) {
                int hh = h + dh - 1, ww = w + dw - 1;
                if (hh < 0 || hh >= H || ww < 0 || ww >= W) continue;
                size_t xi = (((size_t)b * C + c) * H + hh) * W + ww;
                size_t wi = ((size_t)(o * C + c) * 3 + dh) * 3 + dw;
                gw[wi] += g * x[xi];
                gx[xi] += g * wt[wi];
              }
        }
}
