// trsm.cu -- backward substitution R X = Y with the factor's upper triangular
// R (second sub-step of X = R^{-1}(Q^T B), Eq. (qr1), Sec. II-C-4).
//
// The paper's solve runs, for each block of 3 b x b tiles, a triangular solve
// of a diagonal block (Trsm_lunn) and matrix products with the blocks above
// (Gemm_nn_mo), ordered by block rows to keep its disk cache small.  In HBM the
// order is chosen for parallelism instead: blocks of nbt columns are taken
// bottom-up; the diagonal block is solved (one warp per right-hand side) and
// then all rows above are updated at once with a tall dense product
// Y[0:i0] -= R[0:i0, i0:i1] X[i0:i1] that spreads over the whole GPU.
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

// B[0:n, 0:k] <- R^{-1} B[0:n, 0:k]; B is FP64 (b_f64) or FP32.  FP64 B is
// solved in FP64 arithmetic whatever R's storage type; FP32 B (the correction
// solve of the mixed-precision refinement) in FP32.
ct_status launch_trsm(const ct_factor* f, void* B, bool b_f64, int64_t ldb, int64_t k,
                      cudaStream_t s) {
  if (k <= 0 || f->n <= 0) return CT_OK;
  const int64_t n = f->n;
  const int64_t nblk = (n + kTB - 1) / kTB;
  const bool f64 = f->store == CT_F64;
  if (!b_f64 && f64) return CT_ERR_UNSUPPORTED;
  const size_t esz = b_f64 ? 8 : 4;
  for (int64_t blk = nblk - 1; blk >= 0; --blk) {
    const int64_t i0 = blk * kTB;
    const int nbt = (int)(n - i0 < kTB ? n - i0 : kTB);
    const unsigned grid = (unsigned)((k + 7) / 8);
    LaunchScope ls(K_TRSM_DIAG, s, (double)nbt * nbt * k, (double)nbt * nbt * (f64 ? 8 : 4) + 2.0 * nbt * k * esz);
    if (f64)
      k_trsm_diag<double, double, double><<<grid, 256, 0, s>>>((const double*)f->F, f->ld, i0, nbt, (double*)B, ldb, k);
    else if (b_f64)
      k_trsm_diag<float, double, double><<<grid, 256, 0, s>>>((const float*)f->F, f->ld, i0, nbt, (double*)B, ldb, k);
    else
      k_trsm_diag<float, float, float><<<grid, 256, 0, s>>>((const float*)f->F, f->ld, i0, nbt, (float*)B, ldb, k);
    CT_LAUNCH_CHECK();
    if (i0 > 0) {
      const void* Rcol = f64 ? (const void*)((const double*)f->F + i0 * f->ld)
                             : (const void*)((const float*)f->F + i0 * f->ld);
      const void* Xblk = (const char*)B + (size_t)i0 * esz;
      ct_status st = launch_dense_update(Rcol, f64, f->ld, nbt, Xblk, ldb, B, b_f64, ldb, i0, k, s);
      if (st != CT_OK) return st;
    }
  }
  return CT_OK;
}

// B[0:n, 0:k] <- R^{-T} B[0:n, 0:k]: blocks top-down, diagonal forward solve,
// then the rows below get B[i1:n] -= R[i0:i1, i1:n]^T Z.  FP64 B in FP64
// arithmetic; FP32 B (FP32-stored R only) in FP32.
ct_status launch_trsm_t(const ct_factor* f, void* B, bool b_f64, int64_t ldb, int64_t k, cudaStream_t s) {
  if (k <= 0 || f->n <= 0) return CT_OK;
  const int64_t n = f->n;
  const bool f64 = f->store == CT_F64;
  if (!b_f64 && f64) return CT_ERR_UNSUPPORTED;
  const size_t esz = b_f64 ? 8 : 4;
  for (int64_t i0 = 0; i0 < n; i0 += kTB) {
    const int nbt = (int)(n - i0 < kTB ? n - i0 : kTB);
    const unsigned grid = (unsigned)((k + 7) / 8);
    {
      LaunchScope ls(K_TRSM_DIAG, s, (double)nbt * nbt * k, (double)nbt * nbt * (f64 ? 8 : 4) + 2.0 * esz * nbt * k);
      if (f64)
        k_trsm_diag_t<double, double, double><<<grid, 256, 0, s>>>((const double*)f->F, f->ld, i0, nbt, (double*)B, ldb, k);
      else if (b_f64)
        k_trsm_diag_t<float, double, double><<<grid, 256, 0, s>>>((const float*)f->F, f->ld, i0, nbt, (double*)B, ldb, k);
      else
        k_trsm_diag_t<float, float, float><<<grid, 256, 0, s>>>((const float*)f->F, f->ld, i0, nbt, (float*)B, ldb, k);
    }
    CT_LAUNCH_CHECK();
    const int64_t i1 = i0 + nbt;
    if (i1 < n) {
      const void* Rrow = f64 ? (const void*)((const double*)f->F + i0 + i1 * f->ld)
                             : (const void*)((const float*)f->F + i0 + i1 * f->ld);
      ct_status st = launch_dense_update_t(Rrow, f64, f->ld, nbt, (const char*)B + i0 * esz, ldb,
                                           (char*)B + i1 * esz, b_f64, ldb, n - i1, k, s);
      if (st != CT_OK) return st;
    }
  }
  return CT_OK;
}

ct_status launch_rank_check(ct_factor* f, cudaStream_t s) {
  LaunchScope ls(K_RANK, s, 0.0, 2.0 * f->n * (f->store == CT_F64 ? 8 : 4));
  if (f->store == CT_F64) k_rank_check<double><<<1, 1024, 0, s>>>((const double*)f->F, f->ld, f->m, f->n, f->status);
  else k_rank_check<float><<<1, 1024, 0, s>>>((const float*)f->F, f->ld, f->m, f->n, f->status);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

}  // namespace ctqr
