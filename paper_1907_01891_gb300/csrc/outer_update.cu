// outer_update.cu -- the tensor-core trailing update of one 128-column outer
// block of the mixed-precision factorization.
//
// After the inner 32-column panels of an outer block [J, J+nbo) are factored,
// the rest of the matrix C = F[J:m, J+nbo:n] is updated once with the whole
// block reflector Q_J = I - V T V^T of the nbo reflectors:
//   W  = V^T C                  tcgen05 GEMM (split over rows, FP32 partials)
//   W' = T^T W                  here, through the UT-transform form
//                               T^{-1} = S = diag(1/tau) + striu(V^T V): W' solves
//                               S^T W' = W (forward substitution, w'_i = tau_i w_i,
//                               then w_r -= (V^T V)_{ir} w'_i for r > i), which
//                               also covers tau_i = 0 (w'_i = 0);
//   C -= V W'                   tcgen05 GEMM.
// This is the paper's Apply_left_Qt_of_dense_QR with its "S factor"
// (Sec. II-C-3) applied to a 128-column block at once, so C is read and
// written once per 128 columns instead of once per 32.
#include "internal.cuh"

namespace ctqr {
namespace {

constexpr int kNB = 128;

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Vc (column-major, ld ldvc) and Vr (row-major, row stride kNB) get the
// explicit reflectors of the block: V(r, a) = F stored value for r > a, 1 on
// the diagonal, 0 above; columns a >= nbo are zero.  With Vrl != NULL the
// row-major copy is split for error-compensated TF32: Vr = hi part (exact in
// TF32), Vrl = x - hi.
__global__ void __launch_bounds__(256) k_extract_v(const float* __restrict__ F, int64_t ld, int64_t mr,
                                                   int nbo, float* __restrict__ Vc, int64_t ldvc,
                                                   float* __restrict__ Vr, float* __restrict__ Vrl) {
  __shared__ float tile[32][kNB + 1];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  for (int e = threadIdx.x; e < 32 * kNB; e += 256) {
    const int rr = e % 32, a = e / 32;
    const int64_t r = r0 + rr;
    float v = 0.f;
    if (r < mr && a < nbo) v = r > a ? F[r + (int64_t)a * ld] : (r == a ? 1.f : 0.f);
    tile[rr][a] = v;
    if (r < mr) Vc[r + (int64_t)a * ldvc] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * kNB; e += 256) {
    const int a = e % kNB, rr = e / kNB;
    const int64_t r = r0 + rr;
    if (r < mr) {
      const float x = tile[rr][a];
      if (Vrl) {
        const float h = tf32_hi(x);
        Vr[r * kNB + a] = h;
        Vrl[r * kNB + a] = x - h;
      } else {
        Vr[r * kNB + a] = x;
      }
    }
  }
}

// G = V^T V from its split partials: G(i, r) (strict upper part, i < r <
// nbo; zero elsewhere) into Gout[i + r * kNB], one entry per thread, the
// splits added in order with their loads in flight.
__global__ void __launch_bounds__(256) k_reduce_gram(const float* __restrict__ Gp, int gsplits, int64_t gstride,
                                                     int nbo, float* __restrict__ Gout) {
  const int e = blockIdx.x * 256 + threadIdx.x;
  if (e >= kNB * kNB) return;
  const int i = e % kNB, r = e / kNB;
  float s = 0.f;
  if (i < nbo && r < nbo && i < r) {
    int z = 0;
    for (; z + 8 <= gsplits; z += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcg(Gp + (z + u) * gstride + i + (int64_t)r * kNB);
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; z < gsplits; ++z) s += __ldcg(Gp + z * gstride + i + (int64_t)r * kNB);
  }
  Gout[e] = s;
}

// T = S^{-1} for S = diag(1/tau) + striu(G), the compact-WY T of the block's
// nbo reflectors (rows and columns >= nbo are zero).  Block doubling on one
// CTA: T_ii = tau_i (no division, so tau_i = 0 gives H_i = I), then for
// s = 1, 2, ..., 64 and the diagonal block pairs A = [p, p+s), C = [p+s, p+2s):
// T_AC = -T_A S_AC T_C.  T is written column-major, T(i, j) at i + j * kNB.
constexpr int kGS = kNB + 1;  // leading dimension of the 128 x 128 matrices in shared memory
constexpr size_t kTinvSmem = (size_t)3 * kNB * kGS * sizeof(float);

__global__ void __launch_bounds__(256) k_tinv(const float* __restrict__ Gred, const double* __restrict__ tau, int nbo,
                                              float* __restrict__ Tout) {
  extern __shared__ float sm[];
  float* S = sm;              // S(i, j) = G(i, j) for i < j
  float* X = S + kNB * kGS;   // T
  float* Y = X + kNB * kGS;   // S_AC T_C
  const int tid = threadIdx.x;
  for (int e = tid; e < kNB * kNB; e += 256) {
    const int i = e % kNB, j = e / kNB;
    S[i + j * kGS] = __ldcg(Gred + e);
    X[i + j * kGS] = (i == j && i < nbo) ? (float)tau[i] : 0.f;
  }
  __syncthreads();
  for (int s = 1; s < kNB; s *= 2) {
    const int ent = (kNB / (2 * s)) * s * s;
    for (int e = tid; e < ent; e += 256) {
      const int pr = e / (s * s), rr = e % (s * s), r = rr % s, c = rr / s;
      const int p0 = pr * 2 * s, gi = p0 + r, gc = p0 + s + c;
      float acc = 0.f;
      for (int k = 0; k <= c; ++k) acc += S[gi + (p0 + s + k) * kGS] * X[(p0 + s + k) + gc * kGS];
      Y[gi + gc * kGS] = acc;
    }
    __syncthreads();
    for (int e = tid; e < ent; e += 256) {
      const int pr = e / (s * s), rr = e % (s * s), r = rr % s, c = rr / s;
      const int p0 = pr * 2 * s, gi = p0 + r, gc = p0 + s + c;
      float acc = 0.f;
      for (int k = r; k < s; ++k) acc += X[gi + (p0 + k) * kGS] * Y[(p0 + k) + gc * kGS];
      X[gi + gc * kGS] = -acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < kNB * kNB; e += 256) {
    const int i = e % kNB, j = e / kNB;
    Tout[e] = X[i + j * kGS];
  }
}

// W' = T^T sum_z W_z for 64 columns per CTA (the UT-transform solve written as
// a product with the explicit T), split into TF32 high and low parts when Wlo
// is given.  Thread (ty = tid % 16, tx = tid / 16) computes rows ty + 16 i
// (i < 8) and columns tx * 4 + j (j < 4).
constexpr int kTC = 64;
constexpr size_t kApplyTtSmem = (size_t)(kNB * kNB + kNB * kTC) * sizeof(float);

__global__ void __launch_bounds__(256) k_apply_tt(const float* __restrict__ Wp, int wsplits, int64_t wstride,
                                                  const float* __restrict__ T, int64_t nc, float* __restrict__ Wout,
                                                  float* __restrict__ Wlo) {
  extern __shared__ float sm[];
  float* Ts = sm;               // Ts[k * kNB + r] = T(k, r)
  float* Ws = Ts + kNB * kNB;   // Ws[k * kTC + c] = W(k, c0 + c)
  const int tid = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * kTC;
  for (int e0 = tid; e0 < kNB * kNB; e0 += 256 * 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(T + e0 + 256 * u);  // T(k, r) at k + r * kNB
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + 256 * u, k = e % kNB, r = e / kNB;
      Ts[k * kNB + r] = v[u];
    }
  }
  for (int e0 = tid; e0 < kNB * kTC; e0 += 256 * 4) {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    for (int z = 0; z < wsplits; ++z) {
      float w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + 256 * u, k = e % kNB, c = e / kNB;
        w[u] = c0 + c < nc ? __ldcg(Wp + z * wstride + k + (c0 + c) * kNB) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] += w[u];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = e0 + 256 * u, k = e % kNB, c = e / kNB;
      Ws[k * kTC + c] = v[u];
    }
  }
  __syncthreads();
  const int ty = tid % 16, tx = tid / 16;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 4
  for (int k = 0; k < kNB; ++k) {
    float a[8], b[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = Ts[k * kNB + ty + 16 * i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Ws[k * kTC + tx * 4 + j];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t c = c0 + tx * 4 + j;
    if (c >= nc) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t o = ty + 16 * i + c * kNB;
      const float w = acc[i][j];
      if (Wlo) {
        const float h = tf32_hi(w);
        Wout[o] = h;
        Wlo[o] = w - h;
      } else {
        Wout[o] = w;
      }
    }
  }
}

}  // namespace

size_t outer_work_floats(int sms, int64_t m, int64_t n) {
  const int64_t mp = (m + 3) / 4 * 4;
  const int64_t wcols = n > (int64_t)4 * sms * 128 ? n : (int64_t)4 * sms * 128;
  return (size_t)mp * kNB          // Vc
         + (size_t)2 * m * kNB     // Vr (high, low)
         + (size_t)kNB * wcols     // W partials
         + (size_t)2 * kNB * n     // W' (high, low)
         + (size_t)(2 * sms + 2) * kNB * kNB;  // G partials, reduced G, T
}

// Update C = F[J:m, J+nbo:n] with the block reflector of F[J:m, J:J+nbo].
ct_status outer_block_update(ct_factor* f, int64_t J, int nbo, float* work, size_t work_floats, int sms,
                             bool split3, cudaStream_t s, Lookahead* la) {
  const int64_t m = f->m, n = f->n, mr = m - J, nc = n - J - nbo;
  // the previous block's deferred update must be done before C is read
  if (la && la->rest_pending) {
    CT_CUDA_TRY(cudaStreamWaitEvent(s, la->ev_rest, 0));
    la->rest_pending = false;
  }
  if (nc <= 0) return CT_OK;
  float* F = (float*)f->F;
  const int64_t ld = f->ld;
  const int64_t ldvc = (m + 3) / 4 * 4;
  const int64_t wcols = n > (int64_t)4 * sms * 128 ? n : (int64_t)4 * sms * 128;
  float* Vc = work;
  float* Vr = Vc + (size_t)ldvc * kNB;
  float* Vrl = Vr + (size_t)m * kNB;
  float* Wp = Vrl + (size_t)m * kNB;
  float* Wq = Wp + (size_t)kNB * wcols;
  float* Wql = Wq + (size_t)kNB * n;
  float* Gp = Wql + (size_t)kNB * n;
  if (outer_work_floats(sms, m, n) > work_floats) return CT_ERR_INVALID;
  {
    LaunchScope ls(K_COPY, s, 0.0, (double)mr * kNB * 12);
    k_extract_v<<<(unsigned)((mr + 31) / 32), 256, 0, s>>>(F + J + J * ld, ld, mr, nbo, Vc, ldvc, Vr,
                                                           split3 ? Vrl : nullptr);
    CT_LAUNCH_CHECK();
  }
  ct_status st;
  // G = V^T V (128 x 128), split over rows.
  int gs = (int)((mr + 2047) / 2048);
  if (gs > 2 * sms) gs = 2 * sms;
  if (gs < 1) gs = 1;
  if ((st = tc_gemm_tn(Vc, ldvc, Vc, ldvc, kNB, kNB, mr, Gp, kNB, (int64_t)kNB * kNB, 0, gs, split3,
                       f->status, s)) != CT_OK)
    return st;
  // W = V^T C, split over rows when there are too few column tiles.
  const int64_t tiles = (nc + 127) / 128;
  int64_t ws = (2 * sms + tiles - 1) / tiles;
  const int64_t wsmax = (mr + 1023) / 1024;
  if (ws > wsmax) ws = wsmax;
  if (ws * nc > wcols) ws = wcols / nc;
  if (ws < 1) ws = 1;
  float* C = F + J + (J + nbo) * ld;
  if ((st = tc_gemm_tn(Vc, ldvc, C, ld, kNB, nc, mr, Wp, kNB, (int64_t)kNB * nc, 0, (int)ws, split3,
                       f->status, s)) != CT_OK)
    return st;
  // tc_gemm_tn may merge splits: recompute how many partial blocks it wrote.
  {
    int64_t chunk = (mr + ws - 1) / ws;
    chunk = (chunk + 31) / 32 * 32;
    ws = (mr + chunk - 1) / chunk;
    int64_t gchunk = (mr + gs - 1) / gs;
    gchunk = (gchunk + 31) / 32 * 32;
    gs = (int)((mr + gchunk - 1) / gchunk);
  }
  // The reduced G goes to the factor's per-block store (kept for later
  // applications of this block reflector), else into the split area's tail.
  float* Gred = f->Gblk ? f->Gblk + (size_t)(J / kNB) * kNB * kNB : Gp + (size_t)gs * kNB * kNB;
  {
    LaunchScope ls(K_TW, s, (double)kNB * kNB * gs, 4.0 * kNB * kNB * (gs + 1));
    k_reduce_gram<<<kNB * kNB / 256, 256, 0, s>>>(Gp, gs, (int64_t)kNB * kNB, nbo, Gred);
    CT_LAUNCH_CHECK();
  }
  // W' = T^T W: T = S^{-1} once for the block, then one product per 64 columns.
  float* Tb = Gp + (size_t)(2 * sms + 1) * kNB * kNB;
  {
    LaunchScope ls(K_TW, s, (double)kNB * kNB * kNB / 3.0, 8.0 * kNB * kNB);
    static bool attr = false;
    if (!attr) {
      CT_CUDA_TRY(cudaFuncSetAttribute(k_tinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTinvSmem));
      CT_CUDA_TRY(cudaFuncSetAttribute(k_apply_tt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApplyTtSmem));
      attr = true;
    }
    k_tinv<<<1, 256, kTinvSmem, s>>>(Gred, f->tau + J, nbo, Tb);
    CT_LAUNCH_CHECK();
  }
  {
    LaunchScope ls(K_TW, s, 2.0 * kNB * kNB * nc, 4.0 * kNB * nc * (ws + 2));
    k_apply_tt<<<(unsigned)((nc + kTC - 1) / kTC), 256, kApplyTtSmem, s>>>(Wp, (int)ws, (int64_t)kNB * nc, Tb, nc,
                                                                           Wq, split3 ? Wql : nullptr);
    CT_LAUNCH_CHECK();
  }
  // C -= V W'  (A = V stored row-major: kNB x mr column-major with ld kNB),
  // persistent kernel on the pre-split operands.  With look-ahead the next
  // block's kNB columns are updated here and the rest on s2, on all but
  // la->reserve SMs, while the next block's panels proceed on s.
  if (la && la->defer && la->s2 && nc > kNB) {
    if ((st = tc_update_presplit(Vr, Vrl, kNB, Wq, Wql, kNB, mr, kNB, kNB, C, ld, split3, sms, f->status, s)) !=
        CT_OK)
      return st;
    CT_CUDA_TRY(cudaEventRecord(la->ev_w, s));
    CT_CUDA_TRY(cudaStreamWaitEvent(la->s2, la->ev_w, 0));
    st = tc_update_presplit(Vr, Vrl, kNB, Wq + (size_t)kNB * kNB, Wql + (size_t)kNB * kNB, kNB, mr, nc - kNB, kNB,
                            C + (size_t)kNB * ld, ld, split3, sms - la->reserve, f->status, la->s2);
    if (st != CT_OK) return st;
    CT_CUDA_TRY(cudaEventRecord(la->ev_rest, la->s2));
    la->rest_pending = true;
    return CT_OK;
  }
  return tc_update_presplit(Vr, Vrl, kNB, Wq, Wql, kNB, mr, nc, kNB, C, ld, split3, sms, f->status, s);
}

}  // namespace ctqr
