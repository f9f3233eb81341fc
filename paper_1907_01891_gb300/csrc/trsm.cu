// trsm.cu -- backward substitution R X = Y with the factor's upper triangular
// R (second sub-step of X = R^{-1}(Q^T B), Eq. (qr1), Sec. II-C-4).
//
// The paper's solve runs, for each block of 3 b x b tiles, a triangular solve
// of a diagonal block (Trsm_lunn) and matrix products with the blocks above
// (Gemm_nn_mo), ordered by block rows to keep its disk cache small.  In HBM the
// order is chosen for parallelism instead: the rows are halved recursively;
// the bottom half is solved, the top half gets one dense product with it
// (spread over the whole GPU), then the top half is solved; the leaves are
// 64 x 64 diagonal solves (one warp per right-hand side).
#include <math.h>

#include "internal.cuh"

namespace ctqr {

ct_status launch_dense_update(const void* V, bool v_f64, int64_t ldv, int K, const void* W,
                              int64_t ldw, void* C, bool b_f64, int64_t ldc, int64_t mr, int64_t nc,
                              cudaStream_t s);

namespace {

constexpr int kTB = 64;  // diagonal block size

// X[i0:i0+nbt, c] = R[i0:i0+nbt, i0:i0+nbt]^{-1} Y[i0:i0+nbt, c], one warp per
// column c; lane l holds rows l and l+32.  Column-oriented inside the block:
// x_i = y_i / R_ii, then y_r -= R_ri x_i for the rows r < i.
template <typename S, typename TB, typename Acc>
__global__ void __launch_bounds__(256) k_trsm_diag(const S* __restrict__ F, int64_t ld, int64_t i0,
                                                   int nbt, TB* __restrict__ B, int64_t ldb,
                                                   int64_t k) {
  __shared__ Acc Rs[kTB][kTB + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < kTB * kTB; e += 256) {
    const int r = e % kTB, c = e / kTB;
    Rs[r][c] = (r < nbt && c < nbt && r <= c) ? (Acc)F[i0 + r + (i0 + c) * ld] : (Acc)0;
  }
  __syncthreads();
  const int64_t col = (int64_t)blockIdx.x * 8 + warp;
  if (col >= k) return;
  TB* y = B + i0 + col * ldb;
  Acc y0 = lane < nbt ? (Acc)y[lane] : (Acc)0;
  Acc y1 = lane + 32 < nbt ? (Acc)y[lane + 32] : (Acc)0;
  for (int i = nbt - 1; i >= 0; --i) {
    const Acc yi = __shfl_sync(0xffffffffu, i < 32 ? y0 : y1, i & 31);
    const Acc xi = yi / Rs[i][i];
    if (i < 32) {
      if (lane == i) y0 = xi;
    } else if (lane == i - 32) {
      y1 = xi;
    }
    if (lane < i) y0 -= Rs[lane][i] * xi;
    if (lane + 32 < i) y1 -= Rs[lane + 32][i] * xi;
  }
  if (lane < nbt) y[lane] = (TB)y0;
  if (lane + 32 < nbt) y[lane + 32] = (TB)y1;
}

// Z[i0:i0+nbt, c] = R[i0:i0+nbt, i0:i0+nbt]^{-T} Y[i0:i0+nbt, c] (forward
// substitution with the lower triangular R^T), FP64 arithmetic.
template <typename S, typename TB, typename Acc>
__global__ void __launch_bounds__(256) k_trsm_diag_t(const S* __restrict__ F, int64_t ld, int64_t i0,
                                                     int nbt, TB* __restrict__ B, int64_t ldb,
                                                     int64_t k) {
  __shared__ Acc Rs[kTB][kTB + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < kTB * kTB; e += 256) {
    const int r = e % kTB, c = e / kTB;
    Rs[r][c] = (r < nbt && c < nbt && r <= c) ? (Acc)F[i0 + r + (i0 + c) * ld] : (Acc)0;
  }
  __syncthreads();
  const int64_t col = (int64_t)blockIdx.x * 8 + warp;
  if (col >= k) return;
  TB* y = B + i0 + col * ldb;
  Acc y0 = lane < nbt ? (Acc)y[lane] : (Acc)0;
  Acc y1 = lane + 32 < nbt ? (Acc)y[lane + 32] : (Acc)0;
  for (int i = 0; i < nbt; ++i) {
    const Acc yi = __shfl_sync(0xffffffffu, i < 32 ? y0 : y1, i & 31);
    const Acc zi = yi / Rs[i][i];
    if (i < 32) {
      if (lane == i) y0 = zi;
    } else if (lane == i - 32) {
      y1 = zi;
    }
    if (lane > i && lane < nbt) y0 -= Rs[i][lane] * zi;
    if (lane + 32 > i && lane + 32 < nbt) y1 -= Rs[i][lane + 32] * zi;
  }
  if (lane < nbt) y[lane] = (TB)y0;
  if (lane + 32 < nbt) y[lane + 32] = (TB)y1;
}

// Rank / finiteness test on diag(R): CT_ERR_RANK when some
// |R_ii| <= max(m, n) * eps * max_i |R_ii|, CT_ERR_NONFINITE for NaN/Inf.
template <typename S>
__global__ void __launch_bounds__(1024) k_rank_check(const S* __restrict__ F, int64_t ld, int64_t m,
                                                     int64_t n, int* status) {
  __shared__ double s_max[32];
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  if (tid == 0) s_bad = 0;
  double mx = 0.0;
  int nonfinite = 0;
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const double r = fabs((double)F[i + i * ld]);
    if (!isfinite(r)) nonfinite = 1;
    else if (r > mx) mx = r;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) s_max[tid >> 5] = mx;
  __syncthreads();
  if (nonfinite) atomicOr(&s_bad, 2);
  if (tid < 32) {
    double v = tid < (int)(blockDim.x / 32) ? s_max[tid] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (tid == 0) s_max[0] = v;
  }
  __syncthreads();
  const double thr = (double)(m > n ? m : n) * 2.220446049250313e-16 * s_max[0];
  for (int64_t i = tid; i < n; i += blockDim.x) {
    const double r = fabs((double)F[i + i * ld]);
    if (isfinite(r) && !(r > thr)) atomicOr(&s_bad, 1);
  }
  __syncthreads();
  if (tid == 0) {
    if (s_bad & 2) set_status(status, CT_ERR_NONFINITE);
    else if (s_bad & 1) set_status(status, CT_ERR_RANK);
  }
}

}  // namespace

namespace {

struct TrsmCtx {
  const ct_factor* f;
  void* B;
  bool b_f64;
  int64_t ldb, k;
  size_t esz;
  cudaStream_t s;
  const void* R(int64_t r, int64_t c) const {
    return f->store == CT_F64 ? (const void*)((const double*)f->F + r + c * f->ld)
                              : (const void*)((const float*)f->F + r + c * f->ld);
  }
  void* Brow(int64_t r) const { return (char*)B + (size_t)r * esz; }
};

ct_status diag_solve(const TrsmCtx& c, int64_t i0, int nbt, bool transpose) {
  const bool f64 = c.f->store == CT_F64;
  const unsigned grid = (unsigned)((c.k + 7) / 8);
  LaunchScope ls(K_TRSM_DIAG, c.s, (double)nbt * nbt * c.k,
                 (double)nbt * nbt * (f64 ? 8 : 4) + 2.0 * c.esz * nbt * c.k);
  if (!transpose) {
    if (f64)
      k_trsm_diag<double, double, double><<<grid, 256, 0, c.s>>>((const double*)c.f->F, c.f->ld, i0, nbt, (double*)c.B, c.ldb, c.k);
    else if (c.b_f64)
      k_trsm_diag<float, double, double><<<grid, 256, 0, c.s>>>((const float*)c.f->F, c.f->ld, i0, nbt, (double*)c.B, c.ldb, c.k);
    else
      k_trsm_diag<float, float, float><<<grid, 256, 0, c.s>>>((const float*)c.f->F, c.f->ld, i0, nbt, (float*)c.B, c.ldb, c.k);
  } else {
    if (f64)
      k_trsm_diag_t<double, double, double><<<grid, 256, 0, c.s>>>((const double*)c.f->F, c.f->ld, i0, nbt, (double*)c.B, c.ldb, c.k);
    else if (c.b_f64)
      k_trsm_diag_t<float, double, double><<<grid, 256, 0, c.s>>>((const float*)c.f->F, c.f->ld, i0, nbt, (double*)c.B, c.ldb, c.k);
    else
      k_trsm_diag_t<float, float, float><<<grid, 256, 0, c.s>>>((const float*)c.f->F, c.f->ld, i0, nbt, (float*)c.B, c.ldb, c.k);
  }
  CT_LAUNCH_CHECK();
  return CT_OK;
}

// Rows [lo, hi) of R X = B, bottom half first, then the top half gets the
// product with the solved bottom half: B[lo:mid] -= R[lo:mid, mid:hi] X[mid:hi]
// (the Gemm_nn_mo task over a whole block row at once).
ct_status solve_rec(const TrsmCtx& c, int64_t lo, int64_t hi) {
  if (hi - lo <= kTB) return diag_solve(c, lo, (int)(hi - lo), false);
  const int64_t mid = lo + ((hi - lo) / 2 + kTB - 1) / kTB * kTB;
  ct_status st = solve_rec(c, mid, hi);
  if (st != CT_OK) return st;
  st = launch_dense_update(c.R(lo, mid), c.f->store == CT_F64, c.f->ld, (int)(hi - mid), c.Brow(mid), c.ldb,
                           c.Brow(lo), c.b_f64, c.ldb, mid - lo, c.k, c.s);
  if (st != CT_OK) return st;
  return solve_rec(c, lo, mid);
}

// Rows [lo, hi) of R^T Z = B (forward substitution), top half first:
// B[mid:hi] -= R[lo:mid, mid:hi]^T Z[lo:mid].
ct_status solve_rec_t(const TrsmCtx& c, int64_t lo, int64_t hi) {
  if (hi - lo <= kTB) return diag_solve(c, lo, (int)(hi - lo), true);
  const int64_t mid = lo + ((hi - lo) / 2 + kTB - 1) / kTB * kTB;
  ct_status st = solve_rec_t(c, lo, mid);
  if (st != CT_OK) return st;
  st = launch_dense_update_t(c.R(lo, mid), c.f->store == CT_F64, c.f->ld, (int)(mid - lo), c.Brow(lo), c.ldb,
                             c.Brow(mid), c.b_f64, c.ldb, hi - mid, c.k, c.s);
  if (st != CT_OK) return st;
  return solve_rec_t(c, mid, hi);
}

}  // namespace

// B[0:n, 0:k] <- R^{-1} B[0:n, 0:k]; B is FP64 (b_f64) or FP32.  FP64 B is
// solved in FP64 arithmetic whatever R's storage type; FP32 B (the
// preconditioner solves of the mixed-precision refinement) in FP32.
// Recursive halving: 64 x 64 diagonal solves (Trsm_lunn) at the leaves and
// one product per split for the block above (Gemm_nn_mo), so the products
// are few and large instead of one K = 64 update per block column.
ct_status launch_trsm(const ct_factor* f, void* B, bool b_f64, int64_t ldb, int64_t k, cudaStream_t s) {
  if (k <= 0 || f->n <= 0) return CT_OK;
  if (!b_f64 && f->store == CT_F64) return CT_ERR_UNSUPPORTED;
  const TrsmCtx c{f, B, b_f64, ldb, k, (size_t)(b_f64 ? 8 : 4), s};
  return solve_rec(c, 0, f->n);
}

// B[0:n, 0:k] <- R^{-T} B[0:n, 0:k] (same arithmetic rules as launch_trsm).
ct_status launch_trsm_t(const ct_factor* f, void* B, bool b_f64, int64_t ldb, int64_t k, cudaStream_t s) {
  if (k <= 0 || f->n <= 0) return CT_OK;
  if (!b_f64 && f->store == CT_F64) return CT_ERR_UNSUPPORTED;
  const TrsmCtx c{f, B, b_f64, ldb, k, (size_t)(b_f64 ? 8 : 4), s};
  return solve_rec_t(c, 0, f->n);
}

ct_status launch_rank_check(ct_factor* f, cudaStream_t s) {
  LaunchScope ls(K_RANK, s, 0.0, 2.0 * f->n * (f->store == CT_F64 ? 8 : 4));
  if (f->store == CT_F64) k_rank_check<double><<<1, 1024, 0, s>>>((const double*)f->F, f->ld, f->m, f->n, f->status);
  else k_rank_check<float><<<1, 1024, 0, s>>>((const float*)f->F, f->ld, f->m, f->n, f->status);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

}  // namespace ctqr
