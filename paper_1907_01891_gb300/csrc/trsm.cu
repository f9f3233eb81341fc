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
#include <stdlib.h>

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

// ---------------------------------------------------------------------------
// One-launch block substitution for FP32 R and FP32 right-hand sides (the
// preconditioner solves of the mixed-precision refinement, k <= 64).
//
// The recursive scheme above issues about two launches per 64-row block; for
// a few right-hand sides each launch is tiny and the solve is a chain of
// launch latencies.  Here one persistent launch walks 128-row blocks in
// dependency order: a CTA takes the next block row i from a ticket counter
// (bottom-up for R X = B, top-down for R^T Z = B), inverts its diagonal
// block R_ii while the blocks it depends on are still being solved,
// subtracts the product with every finished block X_j as soon as that
// block's flag is set, and forms X_i = R_ii^{-1} Y_i as one more product, so
// that one block of the chain costs two 128 x 128 x k products rather than a
// 128-step substitution.  (Multiplying by the inverted diagonal block trades
// a little accuracy, bounded through the diagonal block's condition number,
// for that parallelism.)  A CTA only waits for blocks whose tickets were
// taken earlier, by CTAs that are running, so the launch always progresses;
// every wait is bounded (2 s, then CT_ERR_TIMEOUT in the status word and the
// CTA leaves).
//
// Work split of a product: thread (r, g) = (tid % 128, tid / 128) holds row
// r of the 128 x 128 block operand for columns [32 g, 32 g + 32) in
// registers and multiplies it with the matching 32 rows of the right-hand
// sides, read from shared memory as broadcasts; the four partial rows are
// then summed in a fixed order.
constexpr int kPB = 64;          // most right-hand sides for the persistent solve
constexpr int kQB = 128;         // block rows
constexpr int kQT = 512;         // threads per CTA
constexpr int kQK = 64;          // right-hand sides per launch (every R block read once for all)
constexpr int kQP = 32;          // right-hand sides per pass of the partial products
constexpr int kQG = kQT / kQB;   // column groups of the block operand (4)
constexpr int kQL = kQB / kQG;   // columns per group (32)
constexpr int kQS = kQB + 1;     // stride of the 128 x 128 shared tiles
constexpr int kXS = kQK + 4;     // stride of the right-hand-side tiles (16-byte rows)
constexpr size_t kQSmemFloats = (size_t)2 * kQB * kQS + (size_t)2 * kQB * kXS;

__device__ __forceinline__ int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_i32(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// X = U^{-1} for the upper triangular 128 x 128 U, both column-major with
// stride kQS in shared memory, by block doubling: the diagonal reciprocals,
// then for s = 1, 2, 4, ... and every pair of diagonal blocks A = [p, p+s),
// C = [p+s, p+2s): X_AC = -X_A (U_AC X_C).  tmp: 4096 floats.
__device__ void tri_inv_f32(const float* __restrict__ U, float* __restrict__ X, float* __restrict__ tmp,
                            int tid) {
  for (int e = tid; e < kQB * kQB; e += kQT) {
    const int rr = e % kQB, cc = e / kQB;
    X[cc * kQS + rr] = rr == cc ? 1.f / U[cc * kQS + cc] : 0.f;
  }
  __syncthreads();
  for (int s = 1; s < kQB; s *= 2) {
    const int ss = s * s, ent = (kQB / (2 * s)) * ss;
    for (int e = tid; e < ent; e += kQT) {
      const int pr = e / ss, rc = e % ss, rr = rc % s, c = rc / s;
      const int p0 = pr * 2 * s, gi = p0 + rr, gc = p0 + s + c;
      float acc = 0.f;
      for (int kk = 0; kk <= c; ++kk)  // X_C is upper triangular
        acc = fmaf(U[(p0 + s + kk) * kQS + gi], X[gc * kQS + p0 + s + kk], acc);
      tmp[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < ent; e += kQT) {
      const int pr = e / ss, rc = e % ss, rr = rc % s, c = rc / s;
      const int p0 = pr * 2 * s, gi = p0 + rr, gc = p0 + s + c;
      float acc = 0.f;
      for (int kk = rr; kk < s; ++kk)  // X_A is upper triangular
        acc = fmaf(X[(p0 + kk) * kQS + gi], tmp[pr * ss + c * s + kk], acc);
      X[gc * kQS + gi] = -acc;
    }
    __syncthreads();
  }
}

// Ps[g][c][r] = sum_u a[u] Y[32 g + u][c] for c < 4 NC4 (zero when the
// thread's operand row is known to be zero).
template <int NC4>
__device__ __forceinline__ void row_partials(const float (&a)[kQL], const float* __restrict__ Y,
                                             float* __restrict__ Ps, int r, int g, bool live) {
  float acc[4 * NC4];
#pragma unroll
  for (int c = 0; c < 4 * NC4; ++c) acc[c] = 0.f;
  if (live) {
#pragma unroll
    for (int u = 0; u < kQL; ++u) {
      const float4* y = reinterpret_cast<const float4*>(Y + (kQL * g + u) * kXS);
#pragma unroll
      for (int q = 0; q < NC4; ++q) {
        const float4 v = y[q];
        acc[4 * q + 0] = fmaf(a[u], v.x, acc[4 * q + 0]);
        acc[4 * q + 1] = fmaf(a[u], v.y, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(a[u], v.z, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(a[u], v.w, acc[4 * q + 3]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4 * NC4; ++c) Ps[(g * kQP + c) * kQB + r] = acc[c];
}

// The four partials of entry (r, c), summed in a fixed order.
__device__ __forceinline__ float sum_parts(const float* __restrict__ Ps, int r, int c) {
  return ((Ps[c * kQB + r] + Ps[(kQP + c) * kQB + r]) + Ps[(2 * kQP + c) * kQB + r]) +
         Ps[(3 * kQP + c) * kQB + r];
}

// NH passes of 4 NC4 right-hand sides each (NH = 2: up to 64 columns, every
// staged R block used for both passes).
template <bool TRANS, int NC4, int NH>
__global__ void __launch_bounds__(kQT, 1) k_trsm_persist(const float* __restrict__ F, int64_t ld, int64_t n,
                                                         float* __restrict__ B, int64_t ldb, int k,
                                                         int* __restrict__ flags, int* __restrict__ ticket,
                                                         int* __restrict__ status) {
  extern __shared__ __align__(16) float psm[];
  float* St = psm;               // a staged 128 x 128 block: op(R)_ij(r, l) at St[l * kQS + r]
  float* Dm = St + kQB * kQS;    // R_ii^{-1} (column-major), then the partial products Ps[g][c][r]
  float* Ps = Dm;
  float* Xs = Dm + kQB * kQS;    // X_j [row][column]
  float* Ys = Xs + kQB * kXS;    // Y_i minus the products so far
  __shared__ int s_t, s_fail;
  const int tid = threadIdx.x, r = tid % kQB, g = tid / kQB;
  const int nb = (int)((n + kQB - 1) / kQB);
  constexpr int kc4 = 4 * NC4 * NH;  // columns carried (>= k)
  for (;;) {
    if (tid == 0) {
      s_t = atomicAdd(ticket, 1);
      s_fail = 0;
    }
    __syncthreads();
    const int t = s_t;
    if (t >= nb) return;
    const int i = TRANS ? t : nb - 1 - t;
    const int64_t i0 = (int64_t)i * kQB;
    const int ni = (int)(n - i0 < kQB ? n - i0 : kQB);
    const int deps = TRANS ? i : nb - 1 - i;

    // R_ii: upper part (the rows below the diagonal hold reflectors), the
    // identity past ni; then its inverse
    for (int e = tid; e < kQB * kQB; e += kQT) {
      const int rr = e % kQB, cc = e / kQB;
      const bool v = rr <= cc && cc < ni;
      cp_async_f32(St + cc * kQS + rr, v ? F + i0 + rr + (i0 + cc) * ld : F, v);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (tid >= ni && tid < kQB) St[tid * kQS + tid] = 1.f;
    __syncthreads();
    tri_inv_f32(St, Dm, Xs, tid);
    // this thread's row of op(R_ii)^{-1}: R_ii^{-1} (upper) or R_ii^{-T} (lower)
    float d[kQL];
#pragma unroll
    for (int u = 0; u < kQL; ++u) d[u] = TRANS ? Dm[r * kQS + kQL * g + u] : Dm[(kQL * g + u) * kQS + r];
    const bool live = TRANS ? (kQL * g <= r) : (kQL * g + kQL - 1 >= r);  // warp-uniform
    __syncthreads();  // Dm and St free
    for (int e = tid; e < kQB * kc4; e += kQT) {
      const int rr = e % kQB, c = e / kQB;
      Ys[rr * kXS + c] = (rr < ni && c < k) ? __ldcg(B + i0 + rr + (int64_t)c * ldb) : 0.f;
    }
    // op(R)_ij for dependency q into St: !TRANS R(i0 + a, j0 + b) = (r, l) = (a, b);
    // TRANS R(j0 + a, i0 + b) = (r, l) = (b, a); a runs along memory
    auto stage = [&](int q) {
      const int j = TRANS ? q : nb - 1 - q;
      const int64_t j0 = (int64_t)j * kQB;
      const int nj = (int)(n - j0 < kQB ? n - j0 : kQB);
      for (int e = tid; e < kQB * kQB; e += kQT) {
        const int a = e % kQB, b = e / kQB;
        const int rr = TRANS ? b : a, l = TRANS ? a : b;
        const bool v = rr < ni && l < nj;
        const float* src = TRANS ? F + j0 + a + (i0 + b) * ld : F + i0 + a + (j0 + b) * ld;
        cp_async_f32(St + l * kQS + rr, v ? src : F, v);
      }
      cp_async_commit();
    };
    if (deps > 0) stage(0);
    for (int q = 0; q < deps; ++q) {
      const int j = TRANS ? q : nb - 1 - q;  // finished blocks first
      const int64_t j0 = (int64_t)j * kQB;
      const int nj = (int)(n - j0 < kQB ? n - j0 : kQB);
      cp_async_wait_all();
      __syncthreads();
      float a[kQL];
#pragma unroll
      for (int u = 0; u < kQL; ++u) a[u] = St[(kQL * g + u) * kQS + r];
      if (tid == 0) {
        const uint64_t start = globaltimer_ns();
        while (ld_acquire_i32(flags + j) == 0) {
          if (ld_volatile_i32(status) != 0) { s_fail = 1; break; }
          if (globaltimer_ns() - start > kBarrierLimitNs) {
            set_status(status, CT_ERR_TIMEOUT);
            s_fail = 1;
            break;
          }
          __nanosleep(32);
        }
      }
      __syncthreads();  // X_j published; St read
      if (s_fail) {
        cp_async_wait_all();
        return;
      }
      for (int e = tid; e < kQB * kc4; e += kQT) {
        const int l = e % kQB, c = e / kQB;
        Xs[l * kXS + c] = (l < nj && c < k) ? __ldcg(B + j0 + l + (int64_t)c * ldb) : 0.f;
      }
      if (q + 1 < deps) stage(q + 1);
      __syncthreads();
#pragma unroll 1
      for (int h = 0; h < NH; ++h) {
        if (h > 0) __syncthreads();  // the previous pass's partials are consumed
        row_partials<NC4>(a, Xs + h * kQP, Ps, r, g, true);
        __syncthreads();
        for (int e = tid; e < kQB * 4 * NC4; e += kQT) {
          const int rr = e % kQB, c = e / kQB;
          Ys[rr * kXS + h * kQP + c] -= sum_parts(Ps, rr, c);
        }
      }
    }
    __syncthreads();  // Y_i complete
#pragma unroll 1
    for (int h = 0; h < NH; ++h) {
      row_partials<NC4>(d, Ys + h * kQP, Ps, r, g, live);
      __syncthreads();
      for (int e = tid; e < kQB * 4 * NC4; e += kQT) {
        const int rr = e % kQB, c = h * kQP + e / kQB;
        if (rr < ni && c < k) B[i0 + rr + (int64_t)c * ldb] = sum_parts(Ps, rr, c - h * kQP);
      }
      __syncthreads();
    }
    if (tid == 0) {
      __threadfence();
      st_release_i32(flags + i, 1);
    }
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
namespace {

bool persist_enabled() {
  static const bool on = [] {
    const char* e = getenv("CTQR_TRSM_RECURSIVE");
    return !(e && *e == '1');
  }();
  return on;
}

// One persistent launch per group of up to 64 columns (FP32 R and B).
template <bool TRANS>
const void* persist_kernel(int kc) {
  if (kc <= 8) return (const void*)k_trsm_persist<TRANS, 2, 1>;
  if (kc <= 16) return (const void*)k_trsm_persist<TRANS, 4, 1>;
  if (kc <= 32) return (const void*)k_trsm_persist<TRANS, 8, 1>;
  return (const void*)k_trsm_persist<TRANS, 8, 2>;
}

ct_status trsm_persist(const ct_factor* f, float* B, int64_t ldb, int64_t k, bool transpose, cudaStream_t s) {
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  const int nb = (int)((f->n + kQB - 1) / kQB);
  int* flags = nullptr;
  const size_t words = (size_t)nb + 4;
  CT_CUDA_TRY(cudaMallocAsync((void**)&flags, words * sizeof(int), s));
  struct Free { int* p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{flags, s};
  const size_t smem = kQSmemFloats * sizeof(float);
  for (int64_t c0 = 0; c0 < k; c0 += kQK) {
    const int kc = (int)(k - c0 < kQK ? k - c0 : kQK);
    const void* fn = transpose ? persist_kernel<true>(kc) : persist_kernel<false>(kc);
    CT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kQT, smem));
    if (per_sm < 1) return CT_ERR_UNSUPPORTED;
    int grid = di.sms * per_sm;
    if (grid > nb) grid = nb;
    CT_CUDA_TRY(cudaMemsetAsync(flags, 0, words * sizeof(int), s));
    LaunchScope ls(K_TRSM_DIAG, s, (double)f->n * f->n * kc, (double)f->n * f->n * 2.0 + 8.0 * f->n * kc);
    const float* F = (const float*)f->F;
    int64_t ld = f->ld, n = f->n, ldb_ = ldb;
    float* Bc = B + c0 * ldb;
    int kc_ = kc;
    int* ticket = flags + nb;
    int* status = f->status;
    void* args[] = {(void*)&F, (void*)&ld, (void*)&n, (void*)&Bc, (void*)&ldb_, (void*)&kc_,
                    (void*)&flags, (void*)&ticket, (void*)&status};
    CT_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(kQT), args, smem, s));
  }
  return CT_OK;
}

}  // namespace

// B[0:n, 0:k] <- R^{-1} B[0:n, 0:k]; B is FP64 (b_f64) or FP32.  FP64 B is
// solved in FP64 arithmetic whatever R's storage type; FP32 B (the
// preconditioner solves of the mixed-precision refinement) in FP32: up to 64
// columns in one persistent launch (its block-row chain is latency-bound, so
// wider right-hand sides go to the recursive scheme below, whose products
// grow with k; CTQR_TRSM_RECURSIVE=1 always uses the recursive scheme).  Recursive halving: 64 x 64 diagonal solves (Trsm_lunn) at
// the leaves and one product per split for the block above (Gemm_nn_mo), so
// the products are few and large instead of one K = 64 update per block
// column.
ct_status launch_trsm(const ct_factor* f, void* B, bool b_f64, int64_t ldb, int64_t k, cudaStream_t s) {
  if (k <= 0 || f->n <= 0) return CT_OK;
  if (f->F_host) return b_f64 ? ooc_trsm(f, (double*)B, ldb, k, s) : CT_ERR_UNSUPPORTED;
  if (!b_f64 && f->store == CT_F64) return CT_ERR_UNSUPPORTED;
  if (!b_f64 && k <= kPB && persist_enabled()) return trsm_persist(f, (float*)B, ldb, k, false, s);
  const TrsmCtx c{f, B, b_f64, ldb, k, (size_t)(b_f64 ? 8 : 4), s};
  return solve_rec(c, 0, f->n);
}

// B[0:n, 0:k] <- R^{-T} B[0:n, 0:k] (same arithmetic rules as launch_trsm).
ct_status launch_trsm_t(const ct_factor* f, void* B, bool b_f64, int64_t ldb, int64_t k, cudaStream_t s) {
  if (k <= 0 || f->n <= 0) return CT_OK;
  if (f->F_host) return CT_ERR_UNSUPPORTED;
  if (!b_f64 && f->store == CT_F64) return CT_ERR_UNSUPPORTED;
  if (!b_f64 && k <= kPB && persist_enabled()) return trsm_persist(f, (float*)B, ldb, k, true, s);
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
