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

// W' (kNB x nc, ld kNB) from the split partials of W and the reduced
// G = V^T V, one warp per column; lane l holds rows l, l+32, l+64, l+96.
constexpr int kGS = kNB + 1;  // row stride of the Gram matrix in shared memory
constexpr size_t kSolveSmem = (size_t)(kNB * kGS + kNB) * sizeof(float);

__global__ void __launch_bounds__(256) k_solve_st(const float* __restrict__ Wp, int wsplits, int64_t wstride,
                                                  const float* __restrict__ Gred, const double* __restrict__ tau,
                                                  int nbo, int64_t nc, float* __restrict__ Wout,
                                                  float* __restrict__ Wlo) {
  extern __shared__ float sm[];
  float* G = sm;              // G[i * kGS + r] = (V^T V)(i, r), strict upper part
  float* ts = sm + kNB * kGS;
  // stage G, eight loads in flight per thread
  for (int e0 = threadIdx.x; e0 < kNB * kNB; e0 += 256 * 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(Gred + e0 + 256 * u);  // kNB * kNB is a multiple of 2048
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + 256 * u, i = e % kNB, r = e / kNB;
      G[i * kGS + r] = v[u];
    }
  }
  for (int i = threadIdx.x; i < kNB; i += 256) ts[i] = i < nbo ? (float)tau[i] : 0.f;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t c = (int64_t)blockIdx.x * 8 + warp; c < nc; c += (int64_t)gridDim.x * 8) {
    float w[4] = {0.f, 0.f, 0.f, 0.f};
    const float* wc = Wp + lane + c * kNB;
    int z = 0;
    for (; z + 4 <= wsplits; z += 4) {
      float v[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) v[u][q] = __ldcg(wc + (z + u) * wstride + 32 * q);
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] += v[u][q];
    }
    for (; z < wsplits; ++z)
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] += __ldcg(wc + z * wstride + 32 * q);
    for (int i = 0; i < nbo; ++i) {
      const int qi = i >> 5;
      const float src = qi == 0 ? w[0] : (qi == 1 ? w[1] : (qi == 2 ? w[2] : w[3]));
      const float wi = __shfl_sync(0xffffffffu, src, i & 31) * ts[i];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = lane + 32 * q;
        if (r == i) w[q] = wi;
        else if (r > i) w[q] -= G[i * kGS + r] * wi;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t o = lane + 32 * q + c * kNB;
      if (Wlo) {
        const float h = tf32_hi(w[q]);
        Wout[o] = h;
        Wlo[o] = w[q] - h;
      } else {
        Wout[o] = w[q];
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
         + (size_t)(2 * sms + 1) * kNB * kNB;  // G partials, reduced G
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
  {
    LaunchScope ls(K_TW, s, (double)kNB * kNB * nc, 4.0 * kNB * nc * (ws + 1));
    unsigned grid = (unsigned)((nc + 7) / 8);
    if (grid > (unsigned)(4 * sms)) grid = (unsigned)(4 * sms);
    static bool attr = false;
    if (!attr) {
      CT_CUDA_TRY(cudaFuncSetAttribute(k_solve_st, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSolveSmem));
      attr = true;
    }
    k_solve_st<<<grid, 256, kSolveSmem, s>>>(Wp, (int)ws, (int64_t)kNB * nc, Gred, f->tau + J, nbo, nc, Wq,
                                             split3 ? Wql : nullptr);
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
