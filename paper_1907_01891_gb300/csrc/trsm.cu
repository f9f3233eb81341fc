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
// launch latencies.  Here one persistent launch walks the block rows in
// dependency order: a CTA takes the next block row i from a ticket counter
// (bottom-up for R X = B, top-down for R^T Z = B), subtracts the products
// with every finished block X_j as soon as that block's flag is set, solves
// its 64 x 64 diagonal block and publishes X_i with a release store of flag i.
// A CTA only waits for blocks whose tickets were taken earlier, by CTAs that
// are running, so the launch always progresses; every wait is bounded (2 s,
// then CT_ERR_TIMEOUT in the status word and the CTA leaves).
constexpr int kPB = 64;  // block rows and the most right-hand sides per launch

__device__ __forceinline__ int ld_acquire_i32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_i32(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

template <int NC>
__device__ __forceinline__ void block_product(float (*Rs)[kPB + 1], float (*Xs)[kPB + 1], float (*Ys)[kPB + 1],
                                              int k, int tid) {
  const int r4 = (tid % 16) * 4, cgp = tid / 16;
  float acc[4][NC];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int w = 0; w < NC; ++w) acc[a][w] = 0.f;
#pragma unroll 8
  for (int l = 0; l < kPB; ++l) {
    float rv[4], xv[NC];
#pragma unroll
    for (int a = 0; a < 4; ++a) rv[a] = Rs[r4 + a][l];
#pragma unroll
    for (int w = 0; w < NC; ++w) xv[w] = Xs[l][cgp + 16 * w];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int w = 0; w < NC; ++w) acc[a][w] = fmaf(rv[a], xv[w], acc[a][w]);
  }
#pragma unroll
  for (int w = 0; w < NC; ++w)
    if (cgp + 16 * w < k)
#pragma unroll
      for (int a = 0; a < 4; ++a) Ys[r4 + a][cgp + 16 * w] -= acc[a][w];
}

template <bool TRANS>
__global__ void __launch_bounds__(256) k_trsm_persist(const float* __restrict__ F, int64_t ld, int64_t n,
                                                      float* __restrict__ B, int64_t ldb, int k,
                                                      int* __restrict__ flags, int* __restrict__ ticket,
                                                      int* __restrict__ status) {
  extern __shared__ float psm[];
  float (*Rs)[kPB + 1] = (float (*)[kPB + 1])psm;                       // an off-diagonal block, then R_ii
  float (*Xs)[kPB + 1] = (float (*)[kPB + 1])(psm + kPB * (kPB + 1));   // X_j [row][column]
  float (*Ys)[kPB + 1] = (float (*)[kPB + 1])(psm + 2 * kPB * (kPB + 1));  // B_i minus the products so far
  __shared__ int s_t, s_fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (int)((n + kPB - 1) / kPB);
  for (;;) {
    if (tid == 0) {
      s_t = atomicAdd(ticket, 1);
      s_fail = 0;
    }
    __syncthreads();
    const int t = s_t;
    if (t >= nb) return;
    const int i = TRANS ? t : nb - 1 - t;
    const int64_t i0 = (int64_t)i * kPB;
    const int ni = (int)(n - i0 < kPB ? n - i0 : kPB);
    // B_i, and the diagonal block R_ii (upper part) held in registers until
    // the end so that loading it is off the dependency chain
    float dreg[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u, r = e % kPB, c = e / kPB;
      Ys[r][c] = (r < ni && c < k) ? __ldcg(B + i0 + r + c * ldb) : 0.f;
      dreg[u] = (r < ni && c < ni && r <= c) ? F[i0 + r + (i0 + c) * ld] : 0.f;
    }
    const int deps = TRANS ? i : nb - 1 - i;
    // the 64 x 64 block op(R)_{ij} for contribution q, 16 elements per
    // thread held in registers so its loads overlap the previous product:
    // element u is (r, c) = (e % 64, e / 64) of the stored block, e = tid + 256 u
    float rreg[16];
    auto load_r = [&](int q) {
      const int j = TRANS ? q : nb - 1 - q;
      const int64_t j0 = (int64_t)j * kPB;
      const int nj = (int)(n - j0 < kPB ? n - j0 : kPB);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * u, a = e % kPB, b = e / kPB;
        // !TRANS: R(i0 + a, j0 + b); TRANS: R(j0 + a, i0 + b) (contiguous along a)
        const bool ok = TRANS ? (a < nj && b < ni) : (a < ni && b < nj);
        rreg[u] = ok ? __ldcg(TRANS ? F + j0 + a + (i0 + b) * ld : F + i0 + a + (j0 + b) * ld) : 0.f;
      }
    };
    if (deps > 0) load_r(0);
    for (int q = 0; q < deps; ++q) {
      const int j = TRANS ? q : nb - 1 - q;  // finished blocks first
      const int64_t j0 = (int64_t)j * kPB;
      const int nj = (int)(n - j0 < kPB ? n - j0 : kPB);
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
      __syncthreads();
      if (s_fail) return;
      float xreg[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * u, r = e % kPB, c = e / kPB;
        xreg[u] = (r < nj && c < k) ? __ldcg(B + j0 + r + c * ldb) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * u, a = e % kPB, b = e / kPB;
        // Rs[r][c] = op(R)_{ij}(r, c)
        if (TRANS) Rs[b][a] = rreg[u];
        else Rs[a][b] = rreg[u];
        Xs[a][b] = xreg[u];
      }
      __syncthreads();
      if (q + 1 < deps) load_r(q + 1);
      // Ys -= Rs Xs with a 4 x NC register tile per thread: rows
      // 4 * (tid % 16) + 0..3, columns tid / 16 + 16 * w (w < NC, c < k);
      // NC = ceil(k / 16) so that a few right-hand sides cost few products
      switch ((k + 15) / 16) {
        case 1: block_product<1>(Rs, Xs, Ys, k, tid); break;
        case 2: block_product<2>(Rs, Xs, Ys, k, tid); break;
        case 3: block_product<3>(Rs, Xs, Ys, k, tid); break;
        default: block_product<4>(Rs, Xs, Ys, k, tid); break;
      }
      __syncthreads();
    }
    // diagonal block: X_i = R_ii^{-1} Ys (or R_ii^{-T}); one warp per column,
    // with the reciprocals of the diagonal computed once
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u, r = e % kPB, c = e / kPB;
      Rs[r][c] = dreg[u];
    }
    __syncthreads();
    float* rdiag = &Xs[0][0];  // free now
    if (tid < ni) rdiag[tid] = 1.f / Rs[tid][tid];
    __syncthreads();
    // warp w solves columns w and w + 8 (then w + 16, w + 24, ...) in pairs,
    // interleaving the two dependency chains
    for (int c = warp; c < k; c += 16) {
      const bool two = c + 8 < k;
      const int c2 = two ? c + 8 : c;
      float y0 = lane < ni ? Ys[lane][c] : 0.f;
      float y1 = lane + 32 < ni ? Ys[lane + 32][c] : 0.f;
      float u0 = lane < ni ? Ys[lane][c2] : 0.f;
      float u1 = lane + 32 < ni ? Ys[lane + 32][c2] : 0.f;
      if (!TRANS) {
        for (int q = ni - 1; q >= 0; --q) {
          const float rq = rdiag[q];
          const float xq = __shfl_sync(0xffffffffu, q < 32 ? y0 : y1, q & 31) * rq;
          const float zq = __shfl_sync(0xffffffffu, q < 32 ? u0 : u1, q & 31) * rq;
          if (q < 32) {
            if (lane == q) { y0 = xq; u0 = zq; }
          } else if (lane == q - 32) {
            y1 = xq;
            u1 = zq;
          }
          const float ra = Rs[lane][q], rb = Rs[lane + 32][q];
          if (lane < q) { y0 -= ra * xq; u0 -= ra * zq; }
          if (lane + 32 < q) { y1 -= rb * xq; u1 -= rb * zq; }
        }
      } else {
        for (int q = 0; q < ni; ++q) {
          const float rq = rdiag[q];
          const float xq = __shfl_sync(0xffffffffu, q < 32 ? y0 : y1, q & 31) * rq;
          const float zq = __shfl_sync(0xffffffffu, q < 32 ? u0 : u1, q & 31) * rq;
          if (q < 32) {
            if (lane == q) { y0 = xq; u0 = zq; }
          } else if (lane == q - 32) {
            y1 = xq;
            u1 = zq;
          }
          const float ra = Rs[q][lane], rb = Rs[q][lane + 32];
          if (lane > q && lane < ni) { y0 -= ra * xq; u0 -= ra * zq; }
          if (lane + 32 > q && lane + 32 < ni) { y1 -= rb * xq; u1 -= rb * zq; }
        }
      }
      if (lane < ni) B[i0 + lane + c * ldb] = y0;
      if (lane + 32 < ni) B[i0 + lane + 32 + c * ldb] = y1;
      if (two) {
        if (lane < ni) B[i0 + lane + c2 * ldb] = u0;
        if (lane + 32 < ni) B[i0 + lane + 32 + c2 * ldb] = u1;
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release_i32(flags + i, 1);
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
ct_status trsm_persist(const ct_factor* f, float* B, int64_t ldb, int64_t k, bool transpose, cudaStream_t s) {
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  const int nb = (int)((f->n + kPB - 1) / kPB);
  int* flags = nullptr;
  const size_t words = (size_t)nb + 4;
  CT_CUDA_TRY(cudaMallocAsync((void**)&flags, words * sizeof(int), s));
  struct Free { int* p; cudaStream_t s; ~Free() { cudaFreeAsync(p, s); } } fr{flags, s};
  const size_t smem = (size_t)3 * kPB * (kPB + 1) * sizeof(float);
  const void* fn = transpose ? (const void*)k_trsm_persist<true> : (const void*)k_trsm_persist<false>;
  CT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem));
  int grid = di.sms * (per_sm > 0 ? per_sm : 1);
  if (grid > nb) grid = nb;
  for (int64_t c0 = 0; c0 < k; c0 += kPB) {
    const int kc = (int)(k - c0 < kPB ? k - c0 : kPB);
    CT_CUDA_TRY(cudaMemsetAsync(flags, 0, words * sizeof(int), s));
    LaunchScope ls(K_TRSM_DIAG, s, (double)f->n * f->n * kc, (double)f->n * f->n * 2.0 + 8.0 * f->n * kc);
    if (transpose)
      k_trsm_persist<true><<<grid, 256, smem, s>>>((const float*)f->F, f->ld, f->n, B + c0 * ldb, ldb, kc, flags,
                                                flags + nb, f->status);
    else
      k_trsm_persist<false><<<grid, 256, smem, s>>>((const float*)f->F, f->ld, f->n, B + c0 * ldb, ldb, kc, flags,
                                                 flags + nb, f->status);
    CT_LAUNCH_CHECK();
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
  if (!b_f64 && f->store == CT_F64) return CT_ERR_UNSUPPORTED;
  if (!b_f64 && k <= kPB && persist_enabled()) return trsm_persist(f, (float*)B, ldb, k, false, s);
  const TrsmCtx c{f, B, b_f64, ldb, k, (size_t)(b_f64 ? 8 : 4), s};
  return solve_rec(c, 0, f->n);
}

// B[0:n, 0:k] <- R^{-T} B[0:n, 0:k] (same arithmetic rules as launch_trsm).
ct_status launch_trsm_t(const ct_factor* f, void* B, bool b_f64, int64_t ldb, int64_t k, cudaStream_t s) {
  if (k <= 0 || f->n <= 0) return CT_OK;
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
