// gemm_simt.cu -- application of a panel's block reflector on the CUDA cores.
//
// Q_p^T C = (I - V T V^T)^T C = C - V (T^T (V^T C)): the GPU form of the
// paper's Apply_left_Qt_of_dense_QR task (Sec. II-C-3), used for the trailing
// update of the factorization and for Q^T B in the solve.  Three kernels:
//   1. k_vtc     partial products P_s = V^T C over row chunk s (split-K: V^T C
//                has a short output (nbp x nc) and a long contraction (mr));
//   2. k_tw      W' = T^T sum_s P_s, the splits summed in a fixed order so the
//                result is bitwise reproducible;
//   3. k_update  C -= V W' (contraction length nbp <= 64).
// V is the unit lower trapezoid stored below the panel's diagonal: V(r, a) =
// stored value for r > a, 1 for r == a, 0 above.  The same k_update also
// serves the triangular solve (dense V = a block column of R).
// FP64 on GB300 runs at ~1.2 TFLOP/s, so the FP64 instances are bound by the
// FP64 pipe, not by memory; register tiles of 4 x TN per thread suffice.
#include "internal.cuh"

namespace ctqr {

constexpr int kBM = 64;   // rows of V^T (reflectors, padded) / rows of a C tile
constexpr int kBK = 16;   // contraction rows per shared-memory stage
constexpr int kGT = 256;  // threads

// V(r, a) of a unit-lower trapezoid (mask) or a dense block (!mask).
template <typename Acc, typename TV>
__device__ __forceinline__ Acc v_at(const TV* V, int64_t ldv, int64_t r, int a, int64_t rows,
                                    int cols, bool mask) {
  if (r >= rows || a >= cols) return (Acc)0;
  if (mask) {
    if (r < a) return (Acc)0;
    if (r == a) return (Acc)1;
  }
  return (Acc)V[r + a * ldv];
}

// P_s = V^T C over the row chunk of split s (blockIdx.y): BM rows of V^T
// (reflectors, padded) x BN columns of C per CTA, RM = BM / 16 rows and
// TN = BN / 16 columns per thread.
template <typename TV, typename TC, typename Acc, int BN, int BM = kBM, bool CMASK = false>
__global__ void __launch_bounds__(kGT) k_vtc(const TV* __restrict__ V, int64_t ldv, int nbp,
                                              const TC* __restrict__ C, int64_t ldc, int64_t mr,
                                              int64_t nc, int64_t chunk, double* __restrict__ part) {
  constexpr int TN = BN / 16, RM = BM / 16;
  __shared__ Acc Vs[kBK][BM + 1];
  __shared__ Acc Cs[kBK][BN + 1];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int64_t c0 = (int64_t)blockIdx.x * BN;
  const int64_t rbeg = (int64_t)blockIdx.y * chunk;
  const int64_t rend = rbeg + chunk < mr ? rbeg + chunk : mr;
  Acc acc[RM][TN];
#pragma unroll
  for (int i = 0; i < RM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = (Acc)0;

  for (int64_t r0 = rbeg; r0 < rend; r0 += kBK) {
#pragma unroll
    for (int i = 0; i < BM * kBK / kGT; ++i) {
      const int e = tid + kGT * i, a = e / kBK, rr = e % kBK;
      const int64_t r = r0 + rr;
      Vs[rr][a] = r < rend ? v_at<Acc>(V, ldv, r, a, mr, nbp, true) : (Acc)0;
    }
#pragma unroll
    for (int i = 0; i < (BN * kBK + kGT - 1) / kGT; ++i) {
      const int e = tid + kGT * i;
      if (e < BN * kBK) {
        const int c = e / kBK, rr = e % kBK;
        const int64_t r = r0 + rr, cg = c0 + c;
        if (CMASK) Cs[rr][c] = r < rend ? v_at<Acc>(C, ldc, r, (int)cg, mr, (int)nc, true) : (Acc)0;
        else Cs[rr][c] = (r < rend && cg < nc) ? (Acc)C[r + cg * ldc] : (Acc)0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      Acc av[RM], cv[TN];
#pragma unroll
      for (int i = 0; i < RM; ++i) av[i] = Vs[kk][ty * RM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) cv[j] = Cs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += av[i] * cv[j];
    }
    __syncthreads();
  }
  double* out = part + (size_t)blockIdx.y * BM * nc;
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int64_t cg = c0 + tx * TN + j;
    if (cg < nc)
#pragma unroll
      for (int i = 0; i < RM; ++i) out[ty * RM + i + cg * BM] = (double)acc[i][j];
  }
}

// W'(a, c) = sum_{b <= a} T(b, a) * sum_s P_s(b, c); one CTA per column c.
// Warp w sums the splits w, w + 8, w + 16, ... (lane l: rows l and l + 32),
// then the eight warp sums are added in order: a fixed order, so the result
// is bitwise reproducible, with many loads in flight per thread.
template <typename Acc>
__global__ void __launch_bounds__(kGT) k_tw(const double* __restrict__ part, int splits,
                                            int64_t nc, const double* __restrict__ T, int ldt,
                                            int nbp, double* __restrict__ W) {
  constexpr int NW = kGT / 32;
  __shared__ double red[NW][kBM];
  __shared__ double sv[kBM];
  __shared__ Acc Ts[kBM][kBM + 1];  // T(b, a) at Ts[a][b]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c = blockIdx.x;
  for (int e0 = tid; e0 < kBM * kBM; e0 += kGT * 4) {  // four loads in flight per thread
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + kGT * u, b = e % kBM, a = e / kBM;  // kBM * kBM is a multiple of 4 * kGT
      v[u] = (a < nbp && b <= a) ? T[b + (int64_t)a * ldt] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + kGT * u, b = e % kBM, a = e / kBM;
      Ts[a][b] = (Acc)v[u];
    }
  }
  const double* base = part + (size_t)c * kBM;
  const size_t stride = (size_t)kBM * nc;
  double s0 = 0.0, s1 = 0.0;
  int sp = warp;
  for (; sp + 3 * NW < splits; sp += 4 * NW) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      v[2 * u] = __ldcg(base + (size_t)(sp + u * NW) * stride + lane);
      v[2 * u + 1] = __ldcg(base + (size_t)(sp + u * NW) * stride + lane + 32);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      s0 += v[2 * u];
      s1 += v[2 * u + 1];
    }
  }
  for (; sp < splits; sp += NW) {
    s0 += __ldcg(base + (size_t)sp * stride + lane);
    s1 += __ldcg(base + (size_t)sp * stride + lane + 32);
  }
  red[warp][lane] = s0;
  red[warp][lane + 32] = s1;
  __syncthreads();
  if (tid < kBM) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) t += red[w][tid];
    sv[tid] = t;
  }
  __syncthreads();
  if (tid < kBM) {
    const int a = tid;
    Acc t = (Acc)0;
    if (a < nbp)
      for (int b = 0; b <= a; ++b) t += Ts[a][b] * (Acc)sv[b];
    W[a + c * kBM] = (double)t;
  }
}

// Outer-block form of W' = T^T sum_s P_s for a 128-column block reflector
// given through S = T^{-1} = diag(1/tau) + striu(G): W' solves S^T W' = W by
// forward substitution (w'_i = tau_i w_i, then w_r -= G(i, r) w'_i for
// r > i; tau_i = 0 gives w'_i = 0).  One CTA per column c: the eight warps
// sum the splits (fixed order), warp 0 substitutes (lane l: rows l + 32 q).
constexpr int kOB = 128;
template <typename Acc, typename TG = float>
__global__ void __launch_bounds__(kGT) k_solve_blk(const double* __restrict__ part, int splits, int64_t nc,
                                                   const TG* __restrict__ G, const double* __restrict__ tau,
                                                   int nbo, double* __restrict__ W) {
  constexpr int NW = kGT / 32;
  extern __shared__ __align__(16) unsigned char gs_raw[];
  TG* gs = (TG*)gs_raw;  // G(i, r) at gs[i * (kOB + 1) + r]
  __shared__ double red[NW][kOB];
  __shared__ Acc ts[kOB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c = blockIdx.x;
  for (int e0 = tid; e0 < kOB * kOB; e0 += kGT * 8) {  // eight loads in flight per thread
    TG v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(G + e0 + kGT * u);  // kOB * kOB is a multiple of 8 * kGT
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + kGT * u, i = e % kOB, r = e / kOB;
      gs[i * (kOB + 1) + r] = v[u];
    }
  }
  for (int i = tid; i < kOB; i += kGT) ts[i] = i < nbo ? (Acc)tau[i] : (Acc)0;
  const double* base = part + (size_t)c * kOB;
  const size_t stride = (size_t)kOB * nc;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int sp = warp; sp < splits; sp += NW) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = __ldcg(base + (size_t)sp * stride + lane + 32 * q);
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += v[q];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[warp][lane + 32 * q] = s[q];
  __syncthreads();
  if (warp != 0) return;
  Acc w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double t = 0.0;
#pragma unroll
    for (int u = 0; u < NW; ++u) t += red[u][lane + 32 * q];
    w[q] = (Acc)t;
  }
  for (int i = 0; i < nbo; ++i) {
    const int qi = i >> 5;
    const Acc src = qi == 0 ? w[0] : (qi == 1 ? w[1] : (qi == 2 ? w[2] : w[3]));
    const Acc wi = __shfl_sync(0xffffffffu, src, i & 31) * ts[i];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = lane + 32 * q;
      if (r == i) w[q] = wi;
      else if (r > i) w[q] -= (Acc)gs[i * (kOB + 1) + r] * wi;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int r = lane + 32 * q;
    W[r + c * kOB] = r < nbo ? (double)w[q] : 0.0;
  }
}

// C(r, c) -= sum_{a < K} V(r, a) W(a, c); 64 x BN tile per CTA, any K.
// Thread (ty = tid % 16, tx = tid / 16) owns rows r0 + ty + 16 i (i < 4) and
// columns c0 + tx * TN + j, so a warp's accesses to C cover 16 consecutive
// rows of two columns (coalesced, C is column-major).
template <typename TV, typename TW, typename TC, typename Acc, int BN>
__global__ void __launch_bounds__(kGT) k_update(const TV* __restrict__ V, int64_t ldv, int K,
                                                 bool mask, const TW* __restrict__ W,
                                                 int64_t ldw, TC* __restrict__ C, int64_t ldc,
                                                 int64_t mr, int64_t nc) {
  constexpr int TN = BN / 16;
  __shared__ Acc Vs[kBK][kBM + 1];
  __shared__ Acc Ws[kBK][BN + 1];
  const int tid = threadIdx.x, ty = tid % 16, tx = tid / 16;
  const int64_t r0 = (int64_t)blockIdx.x * kBM, c0 = (int64_t)blockIdx.y * BN;
  // this thread's C values, loaded first so their latency overlaps the product
  TC cin[4][TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int64_t cg = c0 + tx * TN + j;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = r0 + ty + 16 * i;
      cin[i][j] = (r < mr && cg < nc) ? C[r + cg * ldc] : (TC)0;
    }
  }
  Acc acc[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = (Acc)0;
  for (int a0 = 0; a0 < K; a0 += kBK) {
#pragma unroll
    for (int i = 0; i < kBM * kBK / kGT; ++i) {
      const int e = tid + kGT * i, r = e % kBM, aa = e / kBM;
      Vs[aa][r] = v_at<Acc>(V, ldv, r0 + r, a0 + aa, mr, K, mask);
    }
#pragma unroll
    for (int i = 0; i < (BN * kBK + kGT - 1) / kGT; ++i) {
      const int e = tid + kGT * i;
      if (e < BN * kBK) {
        const int aa = e % kBK, c = e / kBK;
        const int64_t cg = c0 + c;
        Ws[aa][c] = (a0 + aa < K && cg < nc) ? (Acc)W[a0 + aa + cg * ldw] : (Acc)0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      Acc av[4], wv[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = Vs[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) wv[j] = Ws[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += av[i] * wv[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int64_t cg = c0 + tx * TN + j;
    if (cg >= nc) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = r0 + ty + 16 * i;
      if (r < mr) C[r + cg * ldc] = (TC)((Acc)cin[i][j] - acc[i][j]);
    }
  }
}

// C(r, c) -= sum_{a < K} V(a, r) W(a, c): the transposed-V update of the
// forward substitution with R^T (V = a block row of R, read with a < K its
// rows), 64 x BN tile per CTA.
template <typename TV, typename TB, typename Acc, int BN>
__global__ void __launch_bounds__(kGT) k_update_t(const TV* __restrict__ V, int64_t ldv, int K,
                                                   const TB* __restrict__ W, int64_t ldw,
                                                   TB* __restrict__ C, int64_t ldc, int64_t mr,
                                                   int64_t nc) {
  constexpr int TN = BN / 16;
  __shared__ Acc Vs[kBK][kBM + 1];
  __shared__ Acc Ws[kBK][BN + 1];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int64_t r0 = (int64_t)blockIdx.x * kBM, c0 = (int64_t)blockIdx.y * BN;
  Acc acc[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = (Acc)0;
  for (int a0 = 0; a0 < K; a0 += kBK) {
#pragma unroll
    for (int i = 0; i < kBM * kBK / kGT; ++i) {
      const int e = tid + kGT * i, aa = e % kBK, r = e / kBK;
      const int64_t rg = r0 + r;
      Vs[aa][r] = (rg < mr && a0 + aa < K) ? (Acc)V[a0 + aa + rg * ldv] : (Acc)0;
    }
#pragma unroll
    for (int i = 0; i < (BN * kBK + kGT - 1) / kGT; ++i) {
      const int e = tid + kGT * i;
      if (e < BN * kBK) {
        const int aa = e % kBK, c = e / kBK;
        const int64_t cg = c0 + c;
        Ws[aa][c] = (a0 + aa < K && cg < nc) ? (Acc)W[a0 + aa + cg * ldw] : (Acc)0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      Acc av[4], wv[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = Vs[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) wv[j] = Ws[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += av[i] * wv[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int64_t cg = c0 + tx * TN + j;
    if (cg >= nc) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = r0 + ty * 4 + i;
      if (r < mr) C[r + cg * ldc] = (TB)((Acc)C[r + cg * ldc] - acc[i][j]);
    }
  }
}

// Y(a, c) = sum_r A(r, a) R(r, c) for a < n, c < k (FP64 accumulation): A^T R
// with the long contraction over the m rows; 64 x BN output tile per CTA.
template <typename TA, int BN>
__global__ void __launch_bounds__(kGT) k_gemm_tn(const TA* __restrict__ A, int64_t lda,
                                                 const double* __restrict__ R, int64_t ldr,
                                                 double* __restrict__ Y, int64_t ldy, int64_t m,
                                                 int64_t n, int64_t k) {
  constexpr int TN = BN / 16;
  __shared__ double As[kBK][kBM + 1];
  __shared__ double Rs[kBK][BN + 1];
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  const int64_t a0 = (int64_t)blockIdx.x * kBM, c0 = (int64_t)blockIdx.y * BN;
  double acc[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;
  for (int64_t r0 = 0; r0 < m; r0 += kBK) {
#pragma unroll
    for (int i = 0; i < kBM * kBK / kGT; ++i) {
      const int e = tid + kGT * i, a = e / kBK, rr = e % kBK;
      const int64_t r = r0 + rr, ag = a0 + a;
      As[rr][a] = (r < m && ag < n) ? (double)A[r + ag * lda] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < (BN * kBK + kGT - 1) / kGT; ++i) {
      const int e = tid + kGT * i;
      if (e < BN * kBK) {
        const int c = e / kBK, rr = e % kBK;
        const int64_t r = r0 + rr, cg = c0 + c;
        Rs[rr][c] = (r < m && cg < k) ? R[r + cg * ldr] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      double av[4], rv[TN];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) rv[j] = Rs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += av[i] * rv[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int64_t cg = c0 + tx * TN + j;
    if (cg >= k) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t a = a0 + ty * 4 + i;
      if (a < n) Y[a + cg * ldy] = acc[i][j];
    }
  }
}

size_t reflector_work_elems(int sms, int nbp, int64_t nc) {
  (void)nbp;
  return (size_t)kBM * ((size_t)128 * sms + 2 * (size_t)nc) + 64;
}

namespace {

template <typename TV, typename TC, typename Acc, int BN>
ct_status run_reflector(const ReflectorArgs& a, double* work, size_t work_elems, int sms,
                        cudaStream_t s) {
  const int64_t tiles_n = (a.nc + BN - 1) / BN;
  // split-K over rows: about four CTAs per SM, chunks of at least 64 rows,
  // and the partials must fit the work area
  int64_t splits = (4 * sms + tiles_n - 1) / tiles_n;
  const int64_t max_splits = (a.mr + 63) / 64;
  if (splits > max_splits) splits = max_splits;
  const int64_t fit = (int64_t)(work_elems / ((size_t)kBM * a.nc)) - 1;
  if (splits > fit) splits = fit;
  if (a.max_splits > 0 && splits > a.max_splits) splits = a.max_splits;
  if (splits < 1) splits = 1;
  int64_t chunk = (a.mr + splits - 1) / splits;
  chunk = (chunk + kBK - 1) / kBK * kBK;
  splits = (a.mr + chunk - 1) / chunk;
  if (splits < 1) splits = 1;
  const size_t need = (size_t)splits * kBM * a.nc + (size_t)kBM * a.nc;
  if (need > work_elems) return CT_ERR_INVALID;
  double* part = work;
  double* W = work + (size_t)splits * kBM * a.nc;
  const double mnk = (double)a.mr * a.nbp * a.nc;
  {
    LaunchScope ls(K_VTC, s, 2.0 * mnk,
                   (double)a.mr * a.nc * sizeof(TC) + (double)a.mr * a.nbp * sizeof(TV));
    k_vtc<TV, TC, Acc, BN><<<dim3((unsigned)tiles_n, (unsigned)splits), kGT, 0, s>>>(
        (const TV*)a.V, a.ldv, a.nbp, (const TC*)a.C, a.ldc, a.mr, a.nc, chunk, part);
  }
  {
    LaunchScope ls(K_TW, s, (double)a.nbp * a.nbp * a.nc, (double)(splits + 1) * kBM * a.nc * 8);
    k_tw<Acc><<<(unsigned)a.nc, kGT, 0, s>>>(part, (int)splits, a.nc, a.T, a.ldt, a.nbp, W);
  }
  {
    LaunchScope ls(K_UPDATE, s, 2.0 * mnk,
                   2.0 * a.mr * a.nc * sizeof(TC) + (double)a.mr * a.nbp * sizeof(TV));
    k_update<TV, double, TC, Acc, BN><<<dim3((unsigned)((a.mr + kBM - 1) / kBM), (unsigned)tiles_n), kGT, 0, s>>>(
        (const TV*)a.V, a.ldv, a.nbp, true, W, kBM, (TC*)a.C, a.ldc, a.mr, a.nc);
  }
  CT_LAUNCH_CHECK();
  return CT_OK;
}

template <typename TV, typename TC, typename Acc>
ct_status run_reflector_bn(const ReflectorArgs& a, double* work, size_t work_elems, int sms,
                           cudaStream_t s) {
  if (a.nc <= 16) return run_reflector<TV, TC, Acc, 16>(a, work, work_elems, sms, s);
  return run_reflector<TV, TC, Acc, 64>(a, work, work_elems, sms, s);
}

}  // namespace

ct_status apply_block_reflector(const ReflectorArgs& a, double* work, size_t work_elems, int sms,
                                cudaStream_t s) {
  if (a.mr <= 0 || a.nc <= 0 || a.nbp <= 0) return CT_OK;
  if (a.v_f64 && a.c_f64) return run_reflector_bn<double, double, double>(a, work, work_elems, sms, s);
  if (!a.v_f64 && a.c_f64) return run_reflector_bn<float, double, double>(a, work, work_elems, sms, s);
  if (!a.v_f64 && !a.c_f64) {
    if (a.fp32_math) return run_reflector_bn<float, float, float>(a, work, work_elems, sms, s);
    return run_reflector_bn<float, float, double>(a, work, work_elems, sms, s);
  }
  return CT_ERR_UNSUPPORTED;
}

// C(0:mr, 0:nc) -= V(0:mr, 0:K) W(0:K, 0:nc) with a dense V (the solve's block
// updates and the residual B - A X).  W and C share one element type; V may be
// FP64 or FP32; the products accumulate in FP64 unless fp32_math.
namespace {
template <typename TV, typename TB, typename Acc>
void dense_update_t(const void* V, int64_t ldv, int K, const void* W, int64_t ldw, void* C,
                    int64_t ldc, int64_t mr, int64_t nc, cudaStream_t s) {
  LaunchScope ls(K_UPDATE, s, 2.0 * mr * K * nc,
                 2.0 * mr * nc * sizeof(TB) + (double)mr * K * sizeof(TV) + (double)K * nc * sizeof(TB));
  if (nc <= 16) {
    const dim3 grid((unsigned)((mr + kBM - 1) / kBM), (unsigned)((nc + 15) / 16));
    k_update<TV, TB, TB, Acc, 16><<<grid, kGT, 0, s>>>((const TV*)V, ldv, K, false, (const TB*)W, ldw,
                                                       (TB*)C, ldc, mr, nc);
  } else {
    const dim3 grid((unsigned)((mr + kBM - 1) / kBM), (unsigned)((nc + 63) / 64));
    k_update<TV, TB, TB, Acc, 64><<<grid, kGT, 0, s>>>((const TV*)V, ldv, K, false, (const TB*)W, ldw,
                                                       (TB*)C, ldc, mr, nc);
  }
}
}  // namespace

ct_status launch_dense_update(const void* V, bool v_f64, int64_t ldv, int K, const void* W,
                              int64_t ldw, void* C, bool b_f64, int64_t ldc, int64_t mr, int64_t nc,
                              cudaStream_t s) {
  if (mr <= 0 || nc <= 0 || K <= 0) return CT_OK;
  if (b_f64) {
    if (v_f64) dense_update_t<double, double, double>(V, ldv, K, W, ldw, C, ldc, mr, nc, s);
    else dense_update_t<float, double, double>(V, ldv, K, W, ldw, C, ldc, mr, nc, s);
  } else {
    if (v_f64) return CT_ERR_UNSUPPORTED;
    dense_update_t<float, float, float>(V, ldv, K, W, ldw, C, ldc, mr, nc, s);
  }
  CT_LAUNCH_CHECK();
  return CT_OK;
}

namespace {
template <typename TV, typename TB, typename Acc>
void dense_update_t_t(const void* V, int64_t ldv, int K, const void* W, int64_t ldw, void* C, int64_t ldc,
                      int64_t mr, int64_t nc, cudaStream_t s) {
  if (nc <= 16) {
    const dim3 grid((unsigned)((mr + kBM - 1) / kBM), (unsigned)((nc + 15) / 16));
    k_update_t<TV, TB, Acc, 16><<<grid, kGT, 0, s>>>((const TV*)V, ldv, K, (const TB*)W, ldw, (TB*)C, ldc, mr, nc);
  } else {
    const dim3 grid((unsigned)((mr + kBM - 1) / kBM), (unsigned)((nc + 63) / 64));
    k_update_t<TV, TB, Acc, 64><<<grid, kGT, 0, s>>>((const TV*)V, ldv, K, (const TB*)W, ldw, (TB*)C, ldc, mr, nc);
  }
}
}  // namespace

ct_status launch_dense_update_t(const void* V, bool v_f64, int64_t ldv, int K, const void* W, int64_t ldw,
                                void* C, bool b_f64, int64_t ldc, int64_t mr, int64_t nc, cudaStream_t s) {
  if (mr <= 0 || nc <= 0 || K <= 0) return CT_OK;
  LaunchScope ls(K_UPDATE, s, 2.0 * mr * K * nc,
                 (b_f64 ? 16.0 : 8.0) * mr * nc + (double)mr * K * (v_f64 ? 8 : 4));
  if (b_f64) {
    if (v_f64) dense_update_t_t<double, double, double>(V, ldv, K, W, ldw, C, ldc, mr, nc, s);
    else dense_update_t_t<float, double, double>(V, ldv, K, W, ldw, C, ldc, mr, nc, s);
  } else {
    if (v_f64) return CT_ERR_UNSUPPORTED;
    dense_update_t_t<float, float, float>(V, ldv, K, W, ldw, C, ldc, mr, nc, s);
  }
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status launch_gemm_tn(const void* A, bool a_f64, int64_t lda, const double* R, int64_t ldr,
                         double* Y, int64_t ldy, int64_t m, int64_t n, int64_t k, cudaStream_t s) {
  if (m <= 0 || n <= 0 || k <= 0) return CT_OK;
  LaunchScope ls(K_GEMM_TN, s, 2.0 * m * n * k, (double)m * n * (a_f64 ? 8 : 4) + 8.0 * (m + n) * k);
  if (k <= 16) {
    const dim3 grid((unsigned)((n + kBM - 1) / kBM), (unsigned)((k + 15) / 16));
    if (a_f64) k_gemm_tn<double, 16><<<grid, kGT, 0, s>>>((const double*)A, lda, R, ldr, Y, ldy, m, n, k);
    else k_gemm_tn<float, 16><<<grid, kGT, 0, s>>>((const float*)A, lda, R, ldr, Y, ldy, m, n, k);
  } else {
    const dim3 grid((unsigned)((n + kBM - 1) / kBM), (unsigned)((k + 63) / 64));
    if (a_f64) k_gemm_tn<double, 64><<<grid, kGT, 0, s>>>((const double*)A, lda, R, ldr, Y, ldy, m, n, k);
    else k_gemm_tn<float, 64><<<grid, kGT, 0, s>>>((const float*)A, lda, R, ldr, Y, ldy, m, n, k);
  }
  CT_LAUNCH_CHECK();
  return CT_OK;
}

namespace {

// BN: columns of C per CTA (16 for a few right-hand sides; 64 for many, so
// that V is read once per product instead of once per 16 columns).
template <typename TC, typename Acc, int BN>
ct_status run_outer(const ct_factor* f, int64_t J, TC* C, int64_t ldc, int64_t k, double* work, size_t work_elems,
                    int sms, cudaStream_t s) {
  const float* V = (const float*)f->F + J + J * f->ld;
  const int64_t mr = f->m - J;
  const int nbo = kOB;
  const int64_t tiles_n = (k + BN - 1) / BN;
  // splits over rows: about one CTA per SM in all, and the partials (plus W')
  // must fit the work area
  int64_t splits = (sms + tiles_n - 1) / tiles_n;
  const int64_t max_rows = (mr + 255) / 256;
  if (splits > max_rows) splits = max_rows;
  const int64_t fit = (int64_t)(work_elems / ((size_t)kOB * k)) - 1;
  if (splits > fit) splits = fit;
  if (splits < 1) return CT_ERR_INVALID;
  int64_t chunk = (mr + splits - 1) / splits;
  chunk = (chunk + kBK - 1) / kBK * kBK;
  splits = (mr + chunk - 1) / chunk;
  double* part = work;
  double* W = work + (size_t)splits * kOB * k;
  const double mnk = (double)mr * nbo * k;
  {
    LaunchScope ls(K_VTC, s, 2.0 * mnk, (double)mr * k * sizeof(TC) + (double)mr * nbo * 4.0);
    k_vtc<float, TC, Acc, BN, kOB><<<dim3((unsigned)tiles_n, (unsigned)splits), kGT, 0, s>>>(
        V, f->ld, nbo, C, ldc, mr, k, chunk, part);
  }
  {
    const size_t smem = (size_t)kOB * (kOB + 1) * sizeof(float);
    static bool attr = false;
    if (!attr) {
      CT_CUDA_TRY(cudaFuncSetAttribute(k_solve_blk<Acc>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr = true;
    }
    LaunchScope ls(K_TW, s, (double)kOB * kOB * k, (double)(splits + 1) * kOB * k * 8 + smem);
    k_solve_blk<Acc><<<(unsigned)k, kGT, smem, s>>>(part, (int)splits, k, f->Gblk + (size_t)(J / kOB) * kOB * kOB,
                                                    f->tau + J, nbo, W);
  }
  {
    LaunchScope ls(K_UPDATE, s, 2.0 * mnk, 2.0 * mr * k * sizeof(TC) + (double)mr * nbo * 4.0);
    k_update<float, double, TC, Acc, BN><<<dim3((unsigned)((mr + kBM - 1) / kBM), (unsigned)tiles_n), kGT, 0, s>>>(
        V, f->ld, nbo, true, W, kOB, C, ldc, mr, k);
  }
  CT_LAUNCH_CHECK();
  return CT_OK;
}

}  // namespace

namespace {
// G(i, r) = sum_z P_z(i, r) for i, r < nbo (zero elsewhere), 128 x 128 FP64;
// partial z at P + z * 128 * nbo, entry (i, r) at i + r * 128.
__global__ void k_reduce_g64(const double* __restrict__ P, int splits, int nbo, double* __restrict__ G) {
  const int e = blockIdx.x * 256 + threadIdx.x;
  if (e >= kOB * kOB) return;
  const int i = e % kOB, r = e / kOB;
  double acc = 0.0;
  if (i < nbo && r < nbo)
    for (int z = 0; z < splits; ++z) acc += __ldcg(P + (size_t)z * kOB * nbo + i + (size_t)r * kOB);
  G[e] = acc;
}
}  // namespace

size_t fp64_outer_work_elems(int sms, int64_t n) {
  return (size_t)2 * sms * kOB * kOB + (size_t)kOB * kOB + (size_t)kOB * (2 * sms * 64 + 64 + 2 * n);
}

// FP64 two-level factorization: the trailing matrix C = F[J:m, J+nbo:n]
// updated once with the block reflector of the nbo (<= 128) reflectors of
// F[J:m, J:J+nbo], through S = diag(1/tau) + striu(V^T V):
//   G = V^T V (split over rows, reduced), W = V^T C (split-K), W' = S^{-T} W
//   (forward substitution per column), C -= V W'.
// Used when tall panels must be narrow (the panel kernel keeps its rows in
// shared memory), so that the trailing update still contracts over 128.
ct_status fp64_outer_update(ct_factor* f, int64_t J, int nbo, double* work, size_t work_elems, int sms,
                            cudaStream_t s) {
  const int64_t m = f->m, n = f->n, ld = f->ld, mr = m - J, nc = n - J - nbo;
  if (nc <= 0) return CT_OK;
  if (nbo < 1 || nbo > kOB || f->store != CT_F64) return CT_ERR_INVALID;
  if (fp64_outer_work_elems(sms, n) > work_elems) return CT_ERR_INVALID;
  double* V = (double*)f->F + J + J * ld;
  double* C = V + (size_t)nbo * ld;
  double* Gp = work;
  double* G = Gp + (size_t)2 * sms * kOB * kOB;
  double* Wp = G + (size_t)kOB * kOB;
  // 1. G = V^T V
  int64_t gs = (mr + 2047) / 2048;
  if (gs > 2 * sms) gs = 2 * sms;
  if (gs < 1) gs = 1;
  int64_t gchunk = (mr + gs - 1) / gs;
  gchunk = (gchunk + kBK - 1) / kBK * kBK;
  gs = (mr + gchunk - 1) / gchunk;
  {
    LaunchScope ls(K_VTC, s, (double)mr * nbo * nbo, 16.0 * mr * nbo);
    k_vtc<double, double, double, 64, kOB, true><<<dim3((unsigned)((nbo + 63) / 64), (unsigned)gs), kGT, 0, s>>>(
        V, ld, nbo, V, ld, mr, nbo, gchunk, Gp);
    CT_LAUNCH_CHECK();
    k_reduce_g64<<<kOB * kOB / 256, 256, 0, s>>>(Gp, (int)gs, nbo, G);
    CT_LAUNCH_CHECK();
  }
  // 2. W = V^T C, split over rows for about two waves of CTAs
  const int64_t tiles_n = (nc + 63) / 64;
  int64_t splits = (2 * sms + tiles_n - 1) / tiles_n;
  const int64_t max_rows = (mr + 255) / 256;
  if (splits > max_rows) splits = max_rows;
  const int64_t cap = (int64_t)((work_elems - (size_t)(Wp - work)) / ((size_t)kOB * nc)) - 1;
  if (splits > cap) splits = cap;
  if (splits < 1) return CT_ERR_INVALID;
  int64_t chunk = (mr + splits - 1) / splits;
  chunk = (chunk + kBK - 1) / kBK * kBK;
  splits = (mr + chunk - 1) / chunk;
  double* W = Wp + (size_t)splits * kOB * nc;
  const double mnk = (double)mr * nbo * nc;
  {
    LaunchScope ls(K_VTC, s, 2.0 * mnk, 8.0 * ((double)mr * nc + (double)mr * nbo));
    k_vtc<double, double, double, 64, kOB><<<dim3((unsigned)tiles_n, (unsigned)splits), kGT, 0, s>>>(
        V, ld, nbo, C, ld, mr, nc, chunk, Wp);
    CT_LAUNCH_CHECK();
  }
  // 3. W' = S^{-T} W
  {
    const size_t smem = (size_t)kOB * (kOB + 1) * sizeof(double);
    static bool attr = false;
    if (!attr) {
      CT_CUDA_TRY(cudaFuncSetAttribute(k_solve_blk<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
      attr = true;
    }
    LaunchScope ls(K_TW, s, (double)kOB * kOB * nc, (double)(splits + 1) * kOB * nc * 8 + smem);
    k_solve_blk<double, double><<<(unsigned)nc, kGT, smem, s>>>(Wp, (int)splits, nc, G, f->tau + J, nbo, W);
    CT_LAUNCH_CHECK();
  }
  // 4. C -= V W'
  {
    LaunchScope ls(K_UPDATE, s, 2.0 * mnk, 16.0 * mr * nc + 8.0 * mr * nbo);
    k_update<double, double, double, double, 64><<<dim3((unsigned)((mr + kBM - 1) / kBM), (unsigned)tiles_n), kGT, 0,
                                                   s>>>(V, ld, nbo, true, W, kOB, C, ld, mr, nc);
    CT_LAUNCH_CHECK();
  }
  return CT_OK;
}

ct_status apply_outer_reflector(const ct_factor* f, int64_t J, void* C, bool c_f64, int64_t ldc, int64_t k,
                                bool fp32_math, double* work, size_t work_elems, int sms, cudaStream_t s) {
  if (k <= 0) return CT_OK;
  if (!f->Gblk || f->store != CT_F32 || J + kOB > f->n) return CT_ERR_INVALID;
  const bool wide = k >= 48;
  if (c_f64) {
    if (fp32_math)
      return wide ? run_outer<double, float, 64>(f, J, (double*)C, ldc, k, work, work_elems, sms, s)
                  : run_outer<double, float, 16>(f, J, (double*)C, ldc, k, work, work_elems, sms, s);
    return wide ? run_outer<double, double, 64>(f, J, (double*)C, ldc, k, work, work_elems, sms, s)
                : run_outer<double, double, 16>(f, J, (double*)C, ldc, k, work, work_elems, sms, s);
  }
  return wide ? run_outer<float, float, 64>(f, J, (float*)C, ldc, k, work, work_elems, sms, s)
              : run_outer<float, float, 16>(f, J, (float*)C, ldc, k, work, work_elems, sms, s);
}

}  // namespace ctqr
