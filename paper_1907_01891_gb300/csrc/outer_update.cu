// outer_update.cu -- the tensor-core trailing update of one 128-column outer
// block of the mixed-precision factorization, and the one-launch Q^T of all
// outer blocks for FP32 right-hand sides.
//
// After the inner 32-column panels of an outer block [J, J+nbo) are factored,
// the rest of the matrix C = F[J:m, J+nbo:n] is updated once with the whole
// block reflector Q_J = I - V T V^T of the nbo reflectors:
//   G  = V^T V                  tcgen05 GEMM, reduced once and kept per block
//   T  = S^{-1}                 the UT-transform S = diag(1/tau) + striu(G)
//                               inverted by block doubling (T_ii = tau_i, so
//                               tau_i = 0 gives H_i = I), kept per block; on a
//                               side stream beside the next product
//   W  = V^T C                  tcgen05 GEMM (split over rows, FP32 partials)
//   W' = T^T W                  a product per 64 columns (partials summed in order)
//   C -= V W'                   tcgen05 GEMM.
// This is the paper's Apply_left_Qt_of_dense_QR with its "S factor"
// (Sec. II-C-3) applied to a 128-column block at once, so C is read and
// written once per 128 columns instead of once per 32.
#include <cuda_fp16.h>

#include <utility>

#include "internal.cuh"

namespace ctqr {
namespace {

constexpr int kNB = 128;

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Vc (column-major, ld ldvc) and Vr (row-major, row stride W) get the
// explicit reflectors of a block of W columns: V(r, a) = F stored value for
// r > a, 1 on the diagonal, 0 above; columns a >= nbo are zero.  With
// Vrl != NULL the row-major copy is split for error-compensated TF32:
// Vr = hi part (exact in TF32), Vrl = x - hi.
template <int W>
__global__ void __launch_bounds__(256) k_extract_v(const float* __restrict__ F, int64_t ld, int64_t mr,
                                                   int nbo, float* __restrict__ Vc, int64_t ldvc,
                                                   float* __restrict__ Vr, float* __restrict__ Vrl) {
  __shared__ float tile[32][W + 1];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  for (int e = threadIdx.x; e < 32 * W; e += 256) {
    const int rr = e % 32, a = e / 32;
    const int64_t r = r0 + rr;
    float v = 0.f;
    if (r < mr && a < nbo) v = r > a ? F[r + (int64_t)a * ld] : (r == a ? 1.f : 0.f);
    tile[rr][a] = v;
    if (r < mr) Vc[r + (int64_t)a * ldvc] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * W; e += 256) {
    const int a = e % W, rr = e / W;
    const int64_t r = r0 + rr;
    if (r < mr) {
      const float x = tile[rr][a];
      if (Vrl) {
        const float h = tf32_hi(x);
        Vr[r * W + a] = h;
        Vrl[r * W + a] = x - h;
      } else {
        Vr[r * W + a] = x;
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

constexpr int kTinvThreads = 1024;

__global__ void __launch_bounds__(kTinvThreads) k_tinv(const float* __restrict__ Gred, const double* __restrict__ tau,
                                                       int nbo, float* __restrict__ Tout) {
  extern __shared__ float sm[];
  float* S = sm;              // S(i, j) = G(i, j) for i < j
  float* X = S + kNB * kGS;   // T
  float* Y = X + kNB * kGS;   // S_AC T_C
  const int tid = threadIdx.x;
  for (int e = tid; e < kNB * kNB; e += kTinvThreads) {
    const int i = e % kNB, j = e / kNB;
    S[i + j * kGS] = __ldcg(Gred + e);
    X[i + j * kGS] = (i == j && i < nbo) ? (float)tau[i] : 0.f;
  }
  __syncthreads();
  for (int s = 1; s < kNB; s *= 2) {
    const int ent = (kNB / (2 * s)) * s * s;
    for (int e = tid; e < ent; e += kTinvThreads) {
      const int pr = e / (s * s), rr = e % (s * s), r = rr % s, c = rr / s;
      const int p0 = pr * 2 * s, gi = p0 + r, gc = p0 + s + c;
      float acc = 0.f;
      for (int k = 0; k <= c; ++k) acc += S[gi + (p0 + s + k) * kGS] * X[(p0 + s + k) + gc * kGS];
      Y[gi + gc * kGS] = acc;
    }
    __syncthreads();
    for (int e = tid; e < ent; e += kTinvThreads) {
      const int pr = e / (s * s), rr = e % (s * s), r = rr % s, c = rr / s;
      const int p0 = pr * 2 * s, gi = p0 + r, gc = p0 + s + c;
      float acc = 0.f;
      for (int k = r; k < s; ++k) acc += X[gi + (p0 + k) * kGS] * Y[(p0 + k) + gc * kGS];
      X[gi + gc * kGS] = -acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < kNB * kNB; e += kTinvThreads) {
    const int i = e % kNB, j = e / kNB;
    Tout[e] = X[i + j * kGS];
  }
}

// W' = T0^T W[r0 : r0+128] (+ T1^T W[r1 : r1+128] when T1 is given), W the
// sum over the splits z of the partials W_z (rows at stride 1, columns at
// stride ldw), for 64 columns per CTA: the UT-transform solve written as a
// product with the explicit T (two terms for the second half of a 256-column
// block, whose T is [[T_A, T_AB], [0, T_B]]).  Written to Wout (and its TF32
// low part to Wlo when given) with column stride ldo.  Thread (ty = tid % 16,
// tx = tid / 16) computes rows ty + 16 i (i < 8) and columns tx * 4 + j.
constexpr int kTC = 64;
constexpr size_t kApplyTtSmem = (size_t)(kNB * kNB + kNB * kTC) * sizeof(float);

__global__ void __launch_bounds__(256) k_apply_tt(const float* __restrict__ Wp0, int wsplits, int64_t wstride,
                                                  int64_t ldw, const float* __restrict__ T0, int r0,
                                                  const float* __restrict__ T1, int r1, int64_t nc,
                                                  float* __restrict__ Wout, float* __restrict__ Wlo, int64_t ldo) {
  extern __shared__ float sm[];
  float* Ts = sm;               // Ts[k * kNB + r] = T(k, r)
  float* Ws = Ts + kNB * kNB;   // Ws[k * kTC + c] = W(k, c0 + c)
  const int tid = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * kTC;
  const int ty = tid % 16, tx = tid / 16;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 1
  for (int term = 0; term < (T1 ? 2 : 1); ++term) {
  const float* T = term == 0 ? T0 : T1;
  const float* Wp = Wp0 + (term == 0 ? r0 : r1);
  if (term > 0) __syncthreads();  // the previous term's tiles are consumed
  // T: 64 elements per thread, 16 loads in flight at a time
  for (int e0 = tid; e0 < kNB * kNB; e0 += 256 * 16) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = __ldcg(T + e0 + 256 * u);  // T(k, r) at k + r * kNB
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = e0 + 256 * u, k = e % kNB, r = e / kNB;
      Ts[k * kNB + r] = v[u];
    }
  }
  // the W tile summed over the splits in order: 32 elements per thread in two
  // halves, the loads of two splits in flight at a time
#pragma unroll 1
  for (int hv = 0; hv < 2; ++hv) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = 0.f;
    int z = 0;
    for (; z + 2 <= wsplits; z += 2) {
      float w0[16], w1[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * (16 * hv + u), k = e % kNB, c = e / kNB;
        const bool ok = c0 + c < nc;
        w0[u] = ok ? __ldcg(Wp + z * wstride + k + (c0 + c) * ldw) : 0.f;
        w1[u] = ok ? __ldcg(Wp + (z + 1) * wstride + k + (c0 + c) * ldw) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] = (v[u] + w0[u]) + w1[u];
    }
    for (; z < wsplits; ++z) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = tid + 256 * (16 * hv + u), k = e % kNB, c = e / kNB;
        v[u] += c0 + c < nc ? __ldcg(Wp + z * wstride + k + (c0 + c) * ldw) : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * (16 * hv + u), k = e % kNB, c = e / kNB;
      Ws[k * kTC + c] = v[u];
    }
  }
  __syncthreads();
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
  }  // term
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int64_t c = c0 + tx * 4 + j;
    if (c >= nc) continue;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t o = ty + 16 * i + c * ldo;
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


// ---------------------------------------------------------------------------
// Q^T C for the first nblk 128-column outer blocks of a two-level factor in
// one cooperative launch (the solve's Q^T B, FP32 C and arithmetic, k <= 32).
//
// Applying the blocks one by one takes three launches per block whose work
// is a few microseconds each.  Here every CTA owns a fixed range of at most
// kQRC rows of C and keeps them in shared memory for the whole application;
// for block J (reflectors V_J = the unit lower trapezoid of F[J:m, J:J+128],
// compact-WY factor T_J):
//   A. P_c = V_J^T C over the CTA's rows >= J        (partial, to global)
//   -- grid barrier --
//   B. P = sum_c P_c, split over the CTAs, each summing its entries over the
//      partials in a fixed order
//   -- grid barrier --
//   C. W' = T_J^T P (every CTA, from the reduced P), then C -= V_J W' on the
//      CTA's rows.
// The next block's phase A reads only the CTA's own rows, so no barrier is
// needed between C and A.  Thread (a, h) = (tid % 128, tid / 128) forms entry
// a of columns [h KC/2, (h+1) KC/2) in A and C's W' product.
constexpr int kQRC = 160;       // most rows of C a CTA holds
constexpr int kQVS = kQRC + 1;  // column stride of the V slab in shared memory

template <int KC>
constexpr size_t qt_outer_smem_floats() {
  return (size_t)kNB * kQVS + (size_t)kNB * kGS + (size_t)kQRC * (KC + 4) + (size_t)2 * kNB * (KC + 4);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int KC>
__global__ void __launch_bounds__(256, 1) k_qt_outer(const float* __restrict__ F, int64_t ld, int64_t m,
                                                     const float* __restrict__ Tblk, int nblk,
                                                     float* __restrict__ C, int64_t ldc, int k, int rows_per_cta,
                                                     float* __restrict__ part, float* __restrict__ pred,
                                                     unsigned long long* bar, int* status) {
  constexpr int CS = KC + 4;  // row stride of the k-column tiles (16-byte rows)
  constexpr int H = KC / 2;   // columns per thread in the 128-row products
  constexpr int E = kNB * KC; // entries of P
  extern __shared__ __align__(16) float sq[];
  float* Vs = sq;                   // V_J(a_lo + rr, a) at a * kQVS + rr
  float* Ts = Vs + kNB * kQVS;      // T_J(i, a) at a * kGS + i
  float* Cs = Ts + kNB * kGS;       // the CTA's rows of C, [rr][c]
  float* Ps = Cs + kQRC * CS;       // reduced V^T C, [a][c]
  float* Ws = Ps + kNB * CS;        // W', [a][c]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  const int64_t r_lo = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r_hi = r_lo + rows_per_cta < m ? r_lo + rows_per_cta : m;
  const int nrow = r_hi > r_lo ? (int)(r_hi - r_lo) : 0;
  const int c1 = (int)((m + rows_per_cta - 1) / rows_per_cta);  // CTAs that own rows
  for (int e = tid; e < kQRC * KC; e += 256) {
    const int rr = e % kQRC, c = e / kQRC;
    Cs[rr * CS + c] = (rr < nrow && c < k) ? C[r_lo + rr + (int64_t)c * ldc] : 0.f;
  }
  const int a = tid % kNB, h = tid / kNB;
  for (int b = 0; b < nblk; ++b) {
    const int64_t J = (int64_t)b * kNB;
    const int64_t a_lo = r_lo > J ? r_lo : J;
    const int na = r_hi > a_lo ? (int)(r_hi - a_lo) : 0;  // active rows
    const int off = (int)(a_lo - r_lo);
    const int c0 = (int)(J / rows_per_cta);                // first CTA with active rows
    // T_J and the V slab of the active rows (zero above the unit diagonal)
    for (int e = tid; e < kNB * kNB; e += 256)
      cp_async_f32(Ts + (e / kNB) * kGS + (e % kNB), Tblk + (size_t)b * kNB * kNB + e, true);
    for (int e = tid; e < na * kNB; e += 256) {
      const int rr = e % na, col = e / na;
      const int64_t r = a_lo + rr;
      const bool v = r - J > col;
      cp_async_f32(Vs + col * kQVS + rr, v ? F + r + (J + col) * ld : F, v);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (tid < kNB && J + tid >= a_lo && J + tid < r_hi) Vs[tid * kQVS + (int)(J + tid - a_lo)] = 1.f;
    __syncthreads();
    // A. this CTA's V_J^T C
    if (na > 0) {
      float acc[H];
#pragma unroll
      for (int j = 0; j < H; ++j) acc[j] = 0.f;
      for (int rr = 0; rr < na; ++rr) {
        const float v = Vs[a * kQVS + rr];
        const float4* cr = reinterpret_cast<const float4*>(Cs + (off + rr) * CS + h * H);
#pragma unroll
        for (int q = 0; q < H / 4; ++q) {
          const float4 c4 = cr[q];
          acc[4 * q + 0] = fmaf(v, c4.x, acc[4 * q + 0]);
          acc[4 * q + 1] = fmaf(v, c4.y, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(v, c4.z, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(v, c4.w, acc[4 * q + 3]);
        }
      }
#pragma unroll
      for (int j = 0; j < H; ++j) part[((size_t)blockIdx.x * KC + h * H + j) * kNB + a] = acc[j];
    }
    if (!grid_barrier(bar, (unsigned)G, status, kBarrierLimitNs)) return;
    // B. entries [e0, e1) of P summed over the active CTAs' partials
    {
      const int e0 = (int)((int64_t)blockIdx.x * E / G), e1 = (int)((int64_t)(blockIdx.x + 1) * E / G);
      for (int e = e0 + warp; e < e1; e += 8) {
        float s = 0.f;
        for (int z = c0 + lane; z < c1; z += 32) s += __ldcg(part + (size_t)z * E + e);
        s = warp_sum_f(s);
        if (lane == 0) pred[e] = s;
      }
    }
    if (!grid_barrier(bar, (unsigned)G, status, kBarrierLimitNs)) return;
    if (na > 0) {
      for (int e = tid; e < E; e += 256) Ps[(e % kNB) * CS + e / kNB] = __ldcg(pred + e);
      __syncthreads();
      // W'(a, c) = sum_i T(i, a) P(i, c); T is upper triangular, so the sum
      // stops at the warp's last row a
      {
        float acc[H];
#pragma unroll
        for (int j = 0; j < H; ++j) acc[j] = 0.f;
        const int imax = a | 31;
        for (int i = 0; i <= imax; ++i) {
          const float t = Ts[a * kGS + i];
          const float4* pr = reinterpret_cast<const float4*>(Ps + i * CS + h * H);
#pragma unroll
          for (int q = 0; q < H / 4; ++q) {
            const float4 p4 = pr[q];
            acc[4 * q + 0] = fmaf(t, p4.x, acc[4 * q + 0]);
            acc[4 * q + 1] = fmaf(t, p4.y, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(t, p4.z, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(t, p4.w, acc[4 * q + 3]);
          }
        }
#pragma unroll
        for (int j = 0; j < H; ++j) Ws[a * CS + h * H + j] = acc[j];
      }
      __syncthreads();
      // C. C -= V_J W' on the active rows, eight columns per item
      const int items = na * (KC / 8);
      for (int e = tid; e < items; e += 256) {
        const int rr = e % na, g8 = e / na;
        float acc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = 0.f;
        for (int col = 0; col < kNB; ++col) {
          const float v = Vs[col * kQVS + rr];
          const float4* wr = reinterpret_cast<const float4*>(Ws + col * CS + g8 * 8);
          const float4 w0 = wr[0], w1 = wr[1];
          acc[0] = fmaf(v, w0.x, acc[0]);
          acc[1] = fmaf(v, w0.y, acc[1]);
          acc[2] = fmaf(v, w0.z, acc[2]);
          acc[3] = fmaf(v, w0.w, acc[3]);
          acc[4] = fmaf(v, w1.x, acc[4]);
          acc[5] = fmaf(v, w1.y, acc[5]);
          acc[6] = fmaf(v, w1.z, acc[6]);
          acc[7] = fmaf(v, w1.w, acc[7]);
        }
        float* cr = Cs + (off + rr) * CS + g8 * 8;
#pragma unroll
        for (int j = 0; j < 8; ++j) cr[j] -= acc[j];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nrow * KC; e += 256) {
    const int rr = e % nrow, c = e / nrow;
    if (c < k) C[r_lo + rr + (int64_t)c * ldc] = Cs[rr * CS + c];
  }
}

}  // namespace

size_t outer_work_floats(int sms, int64_t m, int64_t n, int width) {
  const int64_t mp = (m + 3) / 4 * 4;
  const int64_t wcols = 8 * n > (int64_t)4 * sms * 128 ? 8 * n : (int64_t)4 * sms * 128;
  const size_t w = width > kNB ? (size_t)width : (size_t)kNB;
  return (size_t)mp * w            // Vc
         + (size_t)2 * m * w       // Vr (high, low)
         + (size_t)w * wcols       // W partials
         + (size_t)2 * w * n       // W' (high, low)
         + (size_t)(2 * sms + 2) * w * w  // G partials, reduced G, T
         + (size_t)3 * kNB * kNB;  // 256-column blocks: reduced G_AB, T_AB, scratch
}

// Update C = F[J:m, J+nbo:cend] with the block reflector of F[J:m, J:J+nbo]
// (cend <= 0: to the last column).
ct_status outer_block_update(ct_factor* f, int64_t J, int nbo, float* work, size_t work_floats, int sms,
                             bool split3, cudaStream_t s, Lookahead* la, int64_t cend) {
  const int64_t m = f->m, n = f->n, mr = m - J, nc = (cend > 0 ? cend : n) - J - nbo;
  // the previous block's deferred update must be done before C is read
  if (la && la->rest_pending) {
    CT_CUDA_TRY(cudaStreamWaitEvent(s, la->ev_rest, 0));
    la->rest_pending = false;
  }
  if (nc <= 0) return CT_OK;
  float* F = (float*)f->F;
  const int64_t ld = f->ld;
  const int64_t ldvc = (m + 3) / 4 * 4;
  const int64_t wcols = 8 * n > (int64_t)4 * sms * 128 ? 8 * n : (int64_t)4 * sms * 128;
  float* Vc = work;
  float* Vr = Vc + (size_t)ldvc * kNB;
  float* Vrl = Vr + (size_t)m * kNB;
  float* Wp = Vrl + (size_t)m * kNB;
  float* Wq = Wp + (size_t)kNB * wcols;
  float* Wql = Wq + (size_t)kNB * n;
  float* Gp = Wql + (size_t)kNB * n;
  if (outer_work_floats(sms, m, n, kNB) > work_floats) return CT_ERR_INVALID;
  if (cend > 0 && la && la->defer) return CT_ERR_INVALID;  // look-ahead updates whole blocks
  {
    LaunchScope ls(K_COPY, s, 0.0, (double)mr * kNB * 12);
    k_extract_v<kNB><<<(unsigned)((mr + 31) / 32), 256, 0, s>>>(F + J + J * ld, ld, mr, nbo, Vc, ldvc, Vr,
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
  // W = V^T C, split over rows when there are too few column tiles: at least
  // two waves of CTAs, and among the split counts up to three times that the
  // one whose last wave is fullest (one CTA per SM; a half-empty last wave
  // costs a whole wave).
  const int64_t tiles = (nc + 127) / 128;
  int64_t wsmax = (mr + 1023) / 1024;
  if (wsmax * nc > wcols) wsmax = wcols / nc;
  if (wsmax < 1) wsmax = 1;
  int64_t ws0 = (2 * sms + tiles - 1) / tiles;
  if (ws0 > wsmax) ws0 = wsmax;
  if (ws0 < 1) ws0 = 1;
  int64_t ws = ws0;
  {
    double best = -1.0;
    for (int64_t w = ws0; w <= 3 * ws0 && w <= wsmax; ++w) {
      // the splits tc_gemm_tn makes of w (chunks rounded up to 32 rows)
      int64_t chunk = (mr + w - 1) / w;
      chunk = (chunk + 31) / 32 * 32;
      const int64_t made = (mr + chunk - 1) / chunk;
      const int64_t ctas = made * tiles;
      const double eff = (double)ctas / (double)(sms * ((ctas + sms - 1) / sms));
      if (eff > best + 0.02) {
        best = eff;
        ws = w;
      }
    }
  }
  // G: the splits tc_gemm_tn wrote (it may merge them)
  {
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
  // T = S^{-1} once for the block (kept in the factor's per-block store, next
  // to G, when there is one), on the side stream beside V^T C when there is one
  float* Tb = f->Tblk ? f->Tblk + (size_t)(J / kNB) * kNB * kNB : Gp + (size_t)(2 * sms + 1) * kNB * kNB;
  const bool side = la && la->s3 && f->Gblk && f->Tblk;
  {
    static bool attr = false;
    if (!attr) {
      CT_CUDA_TRY(cudaFuncSetAttribute(k_tinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTinvSmem));
      CT_CUDA_TRY(cudaFuncSetAttribute(k_apply_tt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApplyTtSmem));
      attr = true;
    }
    cudaStream_t st_t = s;
    if (side) {
      CT_CUDA_TRY(cudaEventRecord(la->ev_g, s));
      CT_CUDA_TRY(cudaStreamWaitEvent(la->s3, la->ev_g, 0));
      st_t = la->s3;
    }
    // (on the side stream its event time includes the wait for a free SM)
    LaunchScope ls(K_TINV, st_t, (double)kNB * kNB * kNB / 3.0, 8.0 * kNB * kNB);
    k_tinv<<<1, kTinvThreads, kTinvSmem, st_t>>>(Gred, f->tau + J, nbo, Tb);
    CT_LAUNCH_CHECK();
    if (side) CT_CUDA_TRY(cudaEventRecord(la->ev_t, la->s3));
  }
  float* C = F + J + (J + nbo) * ld;
  if ((st = tc_gemm_tn(Vc, ldvc, C, ld, kNB, nc, mr, Wp, kNB, (int64_t)kNB * nc, 0, (int)ws, split3,
                       f->status, s)) != CT_OK) {
    if (side) cudaStreamWaitEvent(s, la->ev_t, 0);
    return st;
  }
  // tc_gemm_tn may merge splits: recompute how many partial blocks it wrote.
  {
    int64_t chunk = (mr + ws - 1) / ws;
    chunk = (chunk + 31) / 32 * 32;
    ws = (mr + chunk - 1) / chunk;
  }
  if (side) CT_CUDA_TRY(cudaStreamWaitEvent(s, la->ev_t, 0));
  // W' = T^T W, one product per 64 columns.
  {
    LaunchScope ls(K_TW, s, 2.0 * kNB * kNB * nc, 4.0 * kNB * nc * (ws + 2));
    k_apply_tt<<<(unsigned)((nc + kTC - 1) / kTC), 256, kApplyTtSmem, s>>>(
        Wp, (int)ws, (int64_t)kNB * nc, kNB, Tb, 0, nullptr, 0, nc, Wq, split3 ? Wql : nullptr, kNB);
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

namespace {

// ---------------------------------------------------------------------------
// 256-column outer blocks.  The block reflector of two consecutive 128-column
// halves A = [J, J+128) and B = [J+128, J+256) is I - V T V^T with V = [V_A V_B]
// and T = [[T_A, T_AB], [0, T_B]], T_AB = -T_A (V_A^T V_B) T_B (the compact-WY
// merge of Schreiber and Van Loan).  Updating the trailing matrix once per 256
// columns instead of once per 128 halves the passes over it, the dominant
// HBM traffic of the factorization.
// ---------------------------------------------------------------------------

// out[i + r * ldo] = sum_z P[z * pstride + row0 + i + r * ldp] for i < rows,
// r < cols (the split partials of a tcgen05 product summed in order); with
// strict, entries with i >= r are zero; entries with i >= vr or r >= vc are
// zero.
__global__ void __launch_bounds__(256) k_reduce_block(const float* __restrict__ P, int splits, int64_t pstride,
                                                      int64_t ldp, int row0, int rows, int cols, int vr, int vc,
                                                      int strict, float* __restrict__ out, int64_t ldo) {
  const int e = blockIdx.x * 256 + threadIdx.x;
  if (e >= rows * cols) return;
  const int i = e % rows, r = e / rows;
  float acc = 0.f;
  if (i < vr && r < vc && (!strict || i < r)) {
    const float* p = P + row0 + i + (int64_t)r * ldp;
    int z = 0;
    for (; z + 8 <= splits; z += 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcg(p + (z + u) * pstride);
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += v[u];
    }
    for (; z < splits; ++z) acc += __ldcg(p + z * pstride);
  }
  out[i + (int64_t)r * ldo] = acc;
}

// C = alpha A B for 128 x 128 column-major FP32 matrices (ld 128): the two
// small products of T_AB.  One output per thread, 16 x 16 tiles per CTA.
__global__ void __launch_bounds__(256) k_small_gemm128(const float* __restrict__ A, const float* __restrict__ B,
                                                       float alpha, float* __restrict__ C) {
  __shared__ float As[16][kNB + 1];
  __shared__ float Bs[kNB][17];
  const int ti = threadIdx.x % 16, tj = threadIdx.x / 16;
  const int i0 = blockIdx.x * 16, j0 = blockIdx.y * 16;
  for (int e = threadIdx.x; e < 16 * kNB; e += 256) {
    const int ii = e % 16, k = e / 16;
    As[ii][k] = A[i0 + ii + k * kNB];
  }
  for (int e = threadIdx.x; e < 16 * kNB; e += 256) {
    const int k = e % kNB, jj = e / kNB;
    Bs[k][jj] = B[k + (j0 + jj) * kNB];
  }
  __syncthreads();
  float acc = 0.f;
#pragma unroll 8
  for (int k = 0; k < kNB; ++k) acc = fmaf(As[ti][k], Bs[k][tj], acc);
  C[i0 + ti + (j0 + tj) * kNB] = alpha * acc;
}

}  // namespace

ct_status outer_block_update256(ct_factor* f, int64_t J, int nbo_b, float* work, size_t work_floats, int sms,
                                bool split3, cudaStream_t s, Lookahead* la) {
  constexpr int kW = 2 * kNB;
  const int nbo = kNB + nbo_b;
  const int64_t m = f->m, n = f->n, mr = m - J, nc = n - J - nbo;
  if (nbo_b < 1 || nbo_b > kNB) return CT_ERR_INVALID;
  if (nc <= 0) return CT_OK;
  if (!f->Gblk || !f->Tblk) return CT_ERR_INVALID;
  if (outer_work_floats(sms, m, n, kW) > work_floats) return CT_ERR_INVALID;
  float* F = (float*)f->F;
  const int64_t ld = f->ld;
  const int64_t ldvc = (m + 3) / 4 * 4;
  const int64_t wcols = 8 * n > (int64_t)4 * sms * 128 ? 8 * n : (int64_t)4 * sms * 128;
  float* Vc = work;
  float* Vr = Vc + (size_t)ldvc * kW;
  float* Vrl = Vr + (size_t)m * kW;
  float* Wp = Vrl + (size_t)m * kW;
  float* Wq = Wp + (size_t)kW * wcols;
  float* Wql = Wq + (size_t)kW * n;
  float* Gp = Wql + (size_t)kW * n;
  float* Gab = Gp + (size_t)(2 * sms + 2) * kW * kW;  // reduced V_A^T V_B (128 x 128)
  float* Tab = Gab + (size_t)kNB * kNB;              // T_AB
  float* Ysc = Tab + (size_t)kNB * kNB;              // V_A^T V_B T_B
  {
    LaunchScope ls(K_COPY, s, 0.0, (double)mr * kW * 12);
    k_extract_v<kW><<<(unsigned)((mr + 31) / 32), 256, 0, s>>>(F + J + J * ld, ld, mr, nbo, Vc, ldvc, Vr,
                                                               split3 ? Vrl : nullptr);
    CT_LAUNCH_CHECK();
  }
  ct_status st;
  // [V_A^T V_B; V_B^T V_B] (256 x 128), split over rows.
  int gs = (int)((mr + 2047) / 2048);
  if (gs > 2 * sms) gs = 2 * sms;
  if (gs < 1) gs = 1;
  if ((st = tc_gemm_tn(Vc, ldvc, Vc + (size_t)kNB * ldvc, ldvc, kW, kNB, mr, Gp, kW, (int64_t)kW * kNB, 0, gs,
                       split3, f->status, s)) != CT_OK)
    return st;
  {
    int64_t gchunk = (mr + gs - 1) / gs;
    gchunk = (gchunk + 31) / 32 * 32;
    gs = (int)((mr + gchunk - 1) / gchunk);
  }
  const int64_t hb = J / kNB + 1;  // the second half's index among the 128-column blocks
  float* Gb = f->Gblk + (size_t)hb * kNB * kNB;
  float* Tb = f->Tblk + (size_t)hb * kNB * kNB;
  const float* Ta = f->Tblk + (size_t)(hb - 1) * kNB * kNB;
  {
    LaunchScope ls(K_TW, s, 2.0 * kNB * kNB * gs, 8.0 * kNB * kNB * (gs + 1));
    // G_B = strict upper part of V_B^T V_B; G_AB = V_A^T V_B (all of it)
    k_reduce_block<<<kNB * kNB / 256, 256, 0, s>>>(Gp, gs, (int64_t)kW * kNB, kW, kNB, kNB, kNB, nbo_b, nbo_b, 1,
                                                   Gb, kNB);
    CT_LAUNCH_CHECK();
    k_reduce_block<<<kNB * kNB / 256, 256, 0, s>>>(Gp, gs, (int64_t)kW * kNB, kW, 0, kNB, kNB, kNB, nbo_b, 0,
                                                   Gab, kNB);
    CT_LAUNCH_CHECK();
  }
  // T_B = S_B^{-1}, then T_AB = -T_A (G_AB T_B), on the side stream beside W = V^T C
  const bool side = la && la->s3;
  {
    static bool attr = false;
    if (!attr) {
      CT_CUDA_TRY(cudaFuncSetAttribute(k_tinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTinvSmem));
      CT_CUDA_TRY(cudaFuncSetAttribute(k_apply_tt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApplyTtSmem));
      attr = true;
    }
    cudaStream_t st_t = s;
    if (side) {
      CT_CUDA_TRY(cudaEventRecord(la->ev_g, s));
      CT_CUDA_TRY(cudaStreamWaitEvent(la->s3, la->ev_g, 0));
      st_t = la->s3;
    }
    LaunchScope ls(K_TINV, st_t, (double)kNB * kNB * kNB / 3.0 + 4.0 * kNB * kNB * kNB, 8.0 * kNB * kNB * 4);
    k_tinv<<<1, kTinvThreads, kTinvSmem, st_t>>>(Gb, f->tau + J + kNB, nbo_b, Tb);
    CT_LAUNCH_CHECK();
    k_small_gemm128<<<dim3(kNB / 16, kNB / 16), 256, 0, st_t>>>(Gab, Tb, 1.f, Ysc);
    CT_LAUNCH_CHECK();
    k_small_gemm128<<<dim3(kNB / 16, kNB / 16), 256, 0, st_t>>>(Ta, Ysc, -1.f, Tab);
    CT_LAUNCH_CHECK();
    if (side) CT_CUDA_TRY(cudaEventRecord(la->ev_t, la->s3));
  }
  // W = V^T C (256 x nc), split over rows for full waves of CTAs (two row
  // tiles of V per column tile; they read the same C slices, the second from L2)
  float* C = F + J + (J + nbo) * ld;
  const int64_t tiles = 2 * ((nc + 127) / 128);
  int64_t wsmax = (mr + 1023) / 1024;
  if (wsmax * nc > wcols) wsmax = wcols / nc;
  if (wsmax < 1) wsmax = 1;
  int64_t ws0 = (2 * sms + tiles - 1) / tiles;
  if (ws0 > wsmax) ws0 = wsmax;
  if (ws0 < 1) ws0 = 1;
  int64_t ws = ws0;
  {
    double best = -1.0;
    for (int64_t w = ws0; w <= 3 * ws0 && w <= wsmax; ++w) {
      int64_t chunk = (mr + w - 1) / w;
      chunk = (chunk + 31) / 32 * 32;
      const int64_t made = (mr + chunk - 1) / chunk;
      const int64_t ctas = made * tiles;
      const double eff = (double)ctas / (double)(sms * ((ctas + sms - 1) / sms));
      if (eff > best + 0.02) {
        best = eff;
        ws = w;
      }
    }
  }
  if ((st = tc_gemm_tn(Vc, ldvc, C, ld, kW, nc, mr, Wp, kW, (int64_t)kW * nc, 0, (int)ws, split3, f->status, s)) !=
      CT_OK) {
    if (side) cudaStreamWaitEvent(s, la->ev_t, 0);
    return st;
  }
  {
    int64_t chunk = (mr + ws - 1) / ws;
    chunk = (chunk + 31) / 32 * 32;
    ws = (mr + chunk - 1) / chunk;
  }
  if (side) CT_CUDA_TRY(cudaStreamWaitEvent(s, la->ev_t, 0));
  // W' = T^T W: rows of the first half T_A^T W_A, of the second T_AB^T W_A + T_B^T W_B
  {
    LaunchScope ls(K_TW, s, 2.0 * kW * kNB * nc * 1.5, 4.0 * kW * nc * (ws + 2));
    const unsigned g = (unsigned)((nc + kTC - 1) / kTC);
    k_apply_tt<<<g, 256, kApplyTtSmem, s>>>(Wp, (int)ws, (int64_t)kW * nc, kW, Ta, 0, nullptr, 0, nc, Wq,
                                            split3 ? Wql : nullptr, kW);
    CT_LAUNCH_CHECK();
    k_apply_tt<<<g, 256, kApplyTtSmem, s>>>(Wp, (int)ws, (int64_t)kW * nc, kW, Tab, 0, Tb, kNB, nc, Wq + kNB,
                                            split3 ? Wql + kNB : nullptr, kW);
    CT_LAUNCH_CHECK();
  }
  // C -= V W'  (K = 256)
  return tc_update_presplit(Vr, Vrl, kW, Wq, Wql, kW, mr, nc, kW, C, ld, split3, sms, f->status, s);
}

// Q^T C for the outer blocks [0, nblk) in one cooperative launch; returns
// CT_ERR_UNSUPPORTED (nothing launched) when the factor keeps no T blocks,
// k is outside 1..32, or the rows do not fit kQRC per CTA on this GPU.
ct_status apply_qt_outer_persist(const ct_factor* f, float* C, int64_t ldc, int64_t k, int nblk, double* work,
                                 size_t work_elems, int sms, cudaStream_t s) {
  if (!f->Tblk || f->store != CT_F32 || k < 1 || k > 32 || nblk < 1 || (int64_t)nblk * kNB >= f->n)
    return CT_ERR_UNSUPPORTED;
  const int KC = k <= 16 ? 16 : 32;
  const void* fn = KC == 16 ? (const void*)k_qt_outer<16> : (const void*)k_qt_outer<32>;
  const size_t smem = (KC == 16 ? qt_outer_smem_floats<16>() : qt_outer_smem_floats<32>()) * sizeof(float);
  CT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, smem));
  if (per_sm < 1) return CT_ERR_UNSUPPORTED;
  const int grid = sms * per_sm;
  const int64_t rows = (f->m + grid - 1) / grid;
  if (rows > kQRC) return CT_ERR_UNSUPPORTED;
  // work: partials [grid][KC][128], reduced P [KC][128], barrier counter
  const size_t pfl = (size_t)grid * KC * kNB, rfl = (size_t)KC * kNB;
  const size_t need_bytes = (pfl + rfl) * sizeof(float) + 2 * sizeof(unsigned long long) + 16;
  if (need_bytes > work_elems * sizeof(double)) return CT_ERR_UNSUPPORTED;
  float* part = (float*)work;
  float* pred = part + pfl;
  unsigned long long* bar = (unsigned long long*)(((uintptr_t)(pred + rfl) + 15) & ~(uintptr_t)15);
  CT_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned long long), s));
  const float* F = (const float*)f->F;
  int64_t ld = f->ld, m = f->m, ldc_ = ldc;
  const float* T = f->Tblk;
  int nb_ = nblk, k_ = (int)k, rpc = (int)rows;
  int* status = f->status;
  void* args[] = {(void*)&F, (void*)&ld, (void*)&m, (void*)&T, (void*)&nb_, (void*)&C, (void*)&ldc_, (void*)&k_,
                  (void*)&rpc, (void*)&part, (void*)&pred, (void*)&bar, (void*)&status};
  LaunchScope ls(K_QT_OUTER, s, 4.0 * (double)nblk * kNB * (double)f->m * k,
                 2.0 * (double)nblk * kNB * (double)f->m * 4.0);
  CT_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), args, smem, s));
  return CT_OK;
}

}  // namespace ctqr

namespace ctqr {

// ---------------------------------------------------------------------------
// The same outer-block updates with the operands of the two tensor-core
// products split into two FP16 parts (tc_f16.cu): V scaled by 2^kVExp16, W'
// and the trailing matrix per column.  The trailing matrix's per-column
// scales come from bounds on its columns' magnitudes (F16Cols: column
// 2-norms, which the orthogonal updates keep; the V^T C product of each
// block sums the squares it splits, giving the next block's bounds).
// ---------------------------------------------------------------------------
namespace {

constexpr int kVExp16 = 8;

// Vc16 (column-major, ld ldv) and Vr16 (row-major, row stride W) get the FP16
// parts of the explicit reflectors scaled by 2^kVExp16 (see k_extract_v);
// |v| >= 192 (which would leave FP16's range) is recorded as non-finite.
template <int W>
__global__ void __launch_bounds__(256) k_extract_v16(const float* __restrict__ F, int64_t ld, int64_t mr, int nbo,
                                                     __half* __restrict__ Vch, __half* __restrict__ Vcl, int64_t ldv,
                                                     __half* __restrict__ Vrh, __half* __restrict__ Vrl, int* status) {
  __shared__ float tile[32][W + 1];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const float s = (float)(1 << kVExp16);
  bool bad = false;
  for (int e = threadIdx.x; e < 32 * W; e += 256) {
    const int rr = e % 32, a = e / 32;
    const int64_t r = r0 + rr;
    float v = 0.f;
    if (r < mr && a < nbo) v = r > a ? F[r + (int64_t)a * ld] : (r == a ? 1.f : 0.f);
    bad |= !(fabsf(v) < 192.f);
    tile[rr][a] = v;
    if (r < mr) {
      const float xs = v * s;
      const __half h = __float2half_rn(xs);
      Vch[r + (int64_t)a * ldv] = h;
      Vcl[r + (int64_t)a * ldv] = __float2half_rn(xs - __half2float(h));
    }
  }
  if (bad) set_status(status, CT_ERR_NONFINITE);
  __syncthreads();
  for (int e = threadIdx.x; e < 32 * W; e += 256) {
    const int a = e % W, rr = e / W;
    const int64_t r = r0 + rr;
    if (r < mr) {
      const float xs = tile[rr][a] * s;
      const __half h = __float2half_rn(xs);
      Vrh[r * W + a] = h;
      Vrl[r * W + a] = __float2half_rn(xs - __half2float(h));
    }
  }
}

// T (128 x 128, T(k, r) at k + r * kNB) into Ts[k * kNB + r].
__device__ __forceinline__ void load_t128(const float* __restrict__ T, float* Ts) {
  for (int e0 = threadIdx.x; e0 < kNB * kNB; e0 += 256 * 16) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = __ldcg(T + e0 + 256 * u);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = e0 + 256 * u, k = e % kNB, r = e / kNB;
      Ts[k * kNB + r] = v[u];
    }
  }
}

// Ws[k * kTC + c] = sum_z Wp[z * wstride + k + (c0 + c) * ldw] (k < 128, c < 64,
// the splits added in order; zero beyond nc).
__device__ __forceinline__ void load_w128(const float* __restrict__ Wp, int wsplits, int64_t wstride, int64_t ldw,
                                          int64_t c0, int64_t nc, float* Ws) {
#pragma unroll 1
  for (int hv = 0; hv < 2; ++hv) {
    float v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) v[u] = 0.f;
    for (int z = 0; z < wsplits; ++z) {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int e = threadIdx.x + 256 * (16 * hv + u), k = e % kNB, c = e / kNB;
        v[u] += c0 + c < nc ? __ldcg(Wp + z * wstride + k + (c0 + c) * ldw) : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = threadIdx.x + 256 * (16 * hv + u), k = e % kNB, c = e / kNB;
      Ws[k * kTC + c] = v[u];
    }
  }
}

// acc[i][j] += sum_k Ts[k][ty + 16 i] Ws[k][tx * 4 + j]
__device__ __forceinline__ void tt_product(const float* Ts, const float* Ws, int ty, int tx, float (&acc)[8][4]) {
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
}

// W' = T^T W for 64 columns per CTA and all ROWS rows at once -- ROWS = 128:
// T_A^T W; ROWS = 256: [T_A^T W_A; T_AB^T W_A + T_B^T W_B] -- W summed over
// its split partials.  Each column c is scaled by 2^e_c (its largest |W'|
// below 2^14) and written as FP16 parts Wh + Wl (K x N, column stride ldo);
// winv[c] = 2^-(e_c + kVExp16), the factor the update's epilogue applies.
template <int ROWS>
__global__ void __launch_bounds__(256) k_apply_tt16(const float* __restrict__ Wp, int wsplits, int64_t wstride,
                                                    int64_t ldw, const float* __restrict__ Ta,
                                                    const float* __restrict__ Tab, const float* __restrict__ Tb,
                                                    int64_t nc, __half* __restrict__ Wh, __half* __restrict__ Wl,
                                                    int64_t ldo, float* __restrict__ winv) {
  extern __shared__ float sm[];
  float* Ts = sm;               // Ts[k * kNB + r] = T(k, r)
  float* Ws = Ts + kNB * kNB;   // Ws[k * kTC + c] = W(k, c0 + c)
  const int tid = threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.x * kTC;
  const int ty = tid % 16, tx = tid / 16;
  float top[8][4], bot[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) top[i][j] = bot[i][j] = 0.f;
  load_t128(Ta, Ts);
  load_w128(Wp, wsplits, wstride, ldw, c0, nc, Ws);
  __syncthreads();
  tt_product(Ts, Ws, ty, tx, top);
  if (ROWS == 256) {
    __syncthreads();
    load_t128(Tab, Ts);
    __syncthreads();
    tt_product(Ts, Ws, ty, tx, bot);
    __syncthreads();
    load_t128(Tb, Ts);
    load_w128(Wp + kNB, wsplits, wstride, ldw, c0, nc, Ws);
    __syncthreads();
    tt_product(Ts, Ws, ty, tx, bot);
  }
  // per-column largest |W'| over the ROWS rows: this thread's rows, then the
  // 16 threads (ty) of the column in this half-warp
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) mx = fmaxf(mx, fmaxf(fabsf(top[i][j]), ROWS == 256 ? fabsf(bot[i][j]) : 0.f));
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f && isfinite(mx)) {
      int ex;
      frexpf(mx, &ex);
      e = 14 - ex;
      e = e < -126 ? -126 : (e > 126 ? 126 : e);
    }
    const int64_t c = c0 + tx * 4 + j;
    if (c >= nc) continue;
    const float s = ldexpf(1.f, e);
    if (ty == 0) winv[c] = ldexpf(1.f, -(e + kVExp16));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t o = ty + 16 * i + c * ldo;
      float xs = top[i][j] * s;
      __half h = __float2half_rn(xs);
      Wh[o] = h;
      Wl[o] = __float2half_rn(xs - __half2float(h));
      if (ROWS == 256) {
        xs = bot[i][j] * s;
        h = __float2half_rn(xs);
        Wh[o + kNB] = h;
        Wl[o + kNB] = __float2half_rn(xs - __half2float(h));
      }
    }
  }
}

int64_t up64(int64_t x) { return (x + 63) / 64 * 64; }

// Sub-buffers of the FP16-split update's workspace (offsets in floats, each a
// multiple of 64 floats = 256 bytes).
struct Work16 {
  __half *vch, *vcl, *vrh, *vrl, *wh, *wl;
  float *wp, *winv, *gp, *gab, *tab, *ysc;
  int64_t ldv, wcols;
  size_t total;
};

Work16 carve16(float* base, int sms, int64_t m, int64_t n, int width) {
  Work16 w;
  const int64_t W = width;
  w.ldv = (m + 7) / 8 * 8;
  w.wcols = 8 * n > (int64_t)4 * sms * 128 ? 8 * n : (int64_t)4 * sms * 128;
  int64_t o = 0;
  auto take = [&](int64_t floats) {
    float* p = base ? base + o : nullptr;
    o += up64(floats);
    return p;
  };
  w.vch = (__half*)take(w.ldv * W / 2);
  w.vcl = (__half*)take(w.ldv * W / 2);
  w.vrh = (__half*)take((m * W + 1) / 2);
  w.vrl = (__half*)take((m * W + 1) / 2);
  w.wp = take(W * w.wcols);
  w.wh = (__half*)take((W * n + 1) / 2);
  w.wl = (__half*)take((W * n + 1) / 2);
  w.winv = take(n + 128);  // read by whole 128-column tiles
  w.gp = take((int64_t)(2 * sms + 2) * W * W);
  w.gab = take((int64_t)kNB * kNB);
  w.tab = take((int64_t)kNB * kNB);
  w.ysc = take((int64_t)kNB * kNB);
  w.total = (size_t)o;
  return w;
}

// Split count of W = V^T C over rows: full waves of CTAs, at most wcols / nc
// partial blocks and 1024 rows per split at least (as outer_block_update).
int64_t vtc_splits(int64_t mr, int64_t nc, int64_t wcols, int sms, int m_ctas) {
  const int64_t tiles = m_ctas * ((nc + 127) / 128);
  int64_t wsmax = (mr + 1023) / 1024;
  if (wsmax * nc > wcols) wsmax = wcols / nc;
  if (wsmax < 1) wsmax = 1;
  int64_t ws0 = (2 * sms + tiles - 1) / tiles;
  if (ws0 > wsmax) ws0 = wsmax;
  if (ws0 < 1) ws0 = 1;
  int64_t ws = ws0;
  double best = -1.0;
  for (int64_t w = ws0; w <= 3 * ws0 && w <= wsmax; ++w) {
    int64_t chunk = (mr + w - 1) / w;
    chunk = (chunk + 31) / 32 * 32;
    const int64_t made = (mr + chunk - 1) / chunk;
    const int64_t ctas = made * tiles;
    const double eff = (double)ctas / (double)(sms * ((ctas + sms - 1) / sms));
    if (eff > best + 0.02) {
      best = eff;
      ws = w;
    }
  }
  return ws;
}

constexpr size_t kApplyTt16Smem = (size_t)(kNB * kNB + kNB * kTC) * sizeof(float);

}  // namespace

size_t outer_work_floats16(int sms, int64_t m, int64_t n, int width) {
  return carve16(nullptr, sms, m, n, width).total;
}

ct_status f16_bounds(ct_factor* f, F16Cols* cs, cudaStream_t s) {
  return launch_colnorm_bound((const float*)f->F, f->ld, f->m, f->n, cs->acc, cs->bound, s);
}

// 128-column outer block [J, J + nbo) applied to C = F[J:m, J+nbo:cend] with
// the FP16-split products (cend <= 0: to the last column); cs->bound holds
// bounds on C's column magnitudes.
ct_status outer_update16(ct_factor* f, int64_t J, int nbo, float* work, size_t work_floats, int sms,
                         cudaStream_t s, Lookahead* la, int64_t cend, const F16Cols* cs) {
  const int64_t m = f->m, n = f->n, mr = m - J, nc = (cend > 0 ? cend : n) - J - nbo;
  if (nc <= 0) return CT_OK;
  if (!f->Gblk || !f->Tblk || !cs) return CT_ERR_INVALID;
  const Work16 w = carve16(work, sms, m, n, kNB);
  if (w.total > work_floats) return CT_ERR_INVALID;
  float* F = (float*)f->F;
  const int64_t ld = f->ld;
  {
    LaunchScope ls(K_COPY, s, 0.0, (double)mr * kNB * 12);
    k_extract_v16<kNB><<<(unsigned)((mr + 31) / 32), 256, 0, s>>>(F + J + J * ld, ld, mr, nbo, w.vch, w.vcl, w.ldv,
                                                                   w.vrh, w.vrl, f->status);
    CT_LAUNCH_CHECK();
  }
  ct_status st;
  // G = V^T V (128 x 128), split over rows
  int gs = (int)((mr + 2047) / 2048);
  if (gs > 2 * sms) gs = 2 * sms;
  if (gs < 1) gs = 1;
  const float vinv2 = 1.f / (float)(1 << (2 * kVExp16));
  if ((st = tc_gemm16(w.vch, w.vcl, w.ldv, w.vch, w.vcl, w.ldv, nullptr, nullptr, kNB, kNB, mr, vinv2, w.gp, kNB,
                      (int64_t)kNB * kNB, gs, f->status, s, &gs)) != CT_OK)
    return st;
  float* Gred = f->Gblk + (size_t)(J / kNB) * kNB * kNB;
  {
    LaunchScope ls(K_TW, s, (double)kNB * kNB * gs, 4.0 * kNB * kNB * (gs + 1));
    k_reduce_gram<<<kNB * kNB / 256, 256, 0, s>>>(w.gp, gs, (int64_t)kNB * kNB, nbo, Gred);
    CT_LAUNCH_CHECK();
  }
  float* Tb = f->Tblk + (size_t)(J / kNB) * kNB * kNB;
  const bool side = la && la->s3;
  {
    static bool attr = false;
    if (!attr) {
      CT_CUDA_TRY(cudaFuncSetAttribute(k_tinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTinvSmem));
      CT_CUDA_TRY(cudaFuncSetAttribute(k_apply_tt16<kNB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kApplyTt16Smem));
      CT_CUDA_TRY(cudaFuncSetAttribute(k_apply_tt16<2 * kNB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kApplyTt16Smem));
      attr = true;
    }
    cudaStream_t st_t = s;
    if (side) {
      CT_CUDA_TRY(cudaEventRecord(la->ev_g, s));
      CT_CUDA_TRY(cudaStreamWaitEvent(la->s3, la->ev_g, 0));
      st_t = la->s3;
    }
    LaunchScope ls(K_TINV, st_t, (double)kNB * kNB * kNB / 3.0, 8.0 * kNB * kNB);
    k_tinv<<<1, kTinvThreads, kTinvSmem, st_t>>>(Gred, f->tau + J, nbo, Tb);
    CT_LAUNCH_CHECK();
    if (side) CT_CUDA_TRY(cudaEventRecord(la->ev_t, la->s3));
  }
  // W = V^T C (128 x nc), C split in shared memory with its column scales;
  // for a whole trailing matrix (cend <= 0) the split also sums each
  // column's squares, the next block's bounds
  float* C = F + J + (J + nbo) * ld;
  const bool last = cend <= 0;
  if (last) CT_CUDA_TRY(cudaMemsetAsync(cs->acc + J + nbo, 0, (size_t)nc * sizeof(double), s));
  int ws = (int)vtc_splits(mr, nc, w.wcols, sms, 1);
  if ((st = tc_gemm16(w.vch, w.vcl, w.ldv, C, nullptr, ld, cs->bound + J + nbo, last ? cs->acc + J + nbo : nullptr,
                      kNB, nc, mr, 1.f / (float)(1 << kVExp16), w.wp, kNB, (int64_t)kNB * nc, ws, f->status, s,
                      &ws)) != CT_OK) {
    if (side) cudaStreamWaitEvent(s, la->ev_t, 0);
    return st;
  }
  if (last && (st = launch_norm_bound(cs->acc + J + nbo, nc, cs->bound + J + nbo, s)) != CT_OK) {
    if (side) cudaStreamWaitEvent(s, la->ev_t, 0);
    return st;
  }
  if (side) CT_CUDA_TRY(cudaStreamWaitEvent(s, la->ev_t, 0));
  {
    LaunchScope ls(K_TW, s, 2.0 * kNB * kNB * nc, 4.0 * kNB * nc * (ws + 1));
    k_apply_tt16<kNB><<<(unsigned)((nc + kTC - 1) / kTC), 256, kApplyTt16Smem, s>>>(
        w.wp, ws, (int64_t)kNB * nc, kNB, Tb, nullptr, nullptr, nc, w.wh, w.wl, kNB, w.winv);
    CT_LAUNCH_CHECK();
  }
  return tc_update16(w.vrh, w.vrl, kNB, w.wh, w.wl, kNB, w.winv, mr, nc, kNB, C, ld, sms, f->status, s);
}

// The 256-column update (see outer_block_update256) with the FP16-split
// products; cs->bound holds bounds on the trailing columns' magnitudes.
ct_status outer_update256_16(ct_factor* f, int64_t J, int nbo_b, float* work, size_t work_floats, int sms,
                             cudaStream_t s, Lookahead* la, const F16Cols* cs) {
  constexpr int kW = 2 * kNB;
  const int nbo = kNB + nbo_b;
  const int64_t m = f->m, n = f->n, mr = m - J, nc = n - J - nbo;
  if (nbo_b < 1 || nbo_b > kNB) return CT_ERR_INVALID;
  if (nc <= 0) return CT_OK;
  if (!f->Gblk || !f->Tblk || !cs) return CT_ERR_INVALID;
  const Work16 w = carve16(work, sms, m, n, kW);
  if (w.total > work_floats) return CT_ERR_INVALID;
  float* F = (float*)f->F;
  const int64_t ld = f->ld;
  {
    LaunchScope ls(K_COPY, s, 0.0, (double)mr * kW * 12);
    k_extract_v16<kW><<<(unsigned)((mr + 31) / 32), 256, 0, s>>>(F + J + J * ld, ld, mr, nbo, w.vch, w.vcl, w.ldv,
                                                                  w.vrh, w.vrl, f->status);
    CT_LAUNCH_CHECK();
  }
  ct_status st;
  // [V_A^T V_B; V_B^T V_B] (256 x 128), split over rows
  int gs = (int)((mr + 2047) / 2048);
  if (gs > 2 * sms) gs = 2 * sms;
  if (gs < 1) gs = 1;
  const float vinv2 = 1.f / (float)(1 << (2 * kVExp16));
  if ((st = tc_gemm16(w.vch, w.vcl, w.ldv, w.vch + (size_t)kNB * w.ldv, w.vcl + (size_t)kNB * w.ldv, w.ldv, nullptr,
                      nullptr, kW, kNB, mr, vinv2, w.gp, kW, (int64_t)kW * kNB, gs, f->status, s, &gs)) != CT_OK)
    return st;
  const int64_t hb = J / kNB + 1;
  float* Gb = f->Gblk + (size_t)hb * kNB * kNB;
  float* Tb = f->Tblk + (size_t)hb * kNB * kNB;
  const float* Ta = f->Tblk + (size_t)(hb - 1) * kNB * kNB;
  {
    LaunchScope ls(K_TW, s, 2.0 * kNB * kNB * gs, 8.0 * kNB * kNB * (gs + 1));
    k_reduce_block<<<kNB * kNB / 256, 256, 0, s>>>(w.gp, gs, (int64_t)kW * kNB, kW, kNB, kNB, kNB, nbo_b, nbo_b, 1,
                                                   Gb, kNB);
    CT_LAUNCH_CHECK();
    k_reduce_block<<<kNB * kNB / 256, 256, 0, s>>>(w.gp, gs, (int64_t)kW * kNB, kW, 0, kNB, kNB, kNB, nbo_b, 0,
                                                   w.gab, kNB);
    CT_LAUNCH_CHECK();
  }
  const bool side = la && la->s3;
  {
    static bool attr = false;
    if (!attr) {
      CT_CUDA_TRY(cudaFuncSetAttribute(k_tinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTinvSmem));
      CT_CUDA_TRY(cudaFuncSetAttribute(k_apply_tt16<kNB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kApplyTt16Smem));
      CT_CUDA_TRY(cudaFuncSetAttribute(k_apply_tt16<kW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kApplyTt16Smem));
      attr = true;
    }
    cudaStream_t st_t = s;
    if (side) {
      CT_CUDA_TRY(cudaEventRecord(la->ev_g, s));
      CT_CUDA_TRY(cudaStreamWaitEvent(la->s3, la->ev_g, 0));
      st_t = la->s3;
    }
    LaunchScope ls(K_TINV, st_t, (double)kNB * kNB * kNB / 3.0 + 4.0 * kNB * kNB * kNB, 8.0 * kNB * kNB * 4);
    k_tinv<<<1, kTinvThreads, kTinvSmem, st_t>>>(Gb, f->tau + J + kNB, nbo_b, Tb);
    CT_LAUNCH_CHECK();
    k_small_gemm128<<<dim3(kNB / 16, kNB / 16), 256, 0, st_t>>>(w.gab, Tb, 1.f, w.ysc);
    CT_LAUNCH_CHECK();
    k_small_gemm128<<<dim3(kNB / 16, kNB / 16), 256, 0, st_t>>>(Ta, w.ysc, -1.f, w.tab);
    CT_LAUNCH_CHECK();
    if (side) CT_CUDA_TRY(cudaEventRecord(la->ev_t, la->s3));
  }
  // W = V^T C (256 x nc): each CTA covers both halves' reflectors, so C is
  // read and split once per slice
  float* C = F + J + (J + nbo) * ld;
  CT_CUDA_TRY(cudaMemsetAsync(cs->acc + J + nbo, 0, (size_t)nc * sizeof(double), s));
  int ws = (int)vtc_splits(mr, nc, w.wcols, sms, tc_gemm16_m_ctas(kW));
  if ((st = tc_gemm16(w.vch, w.vcl, w.ldv, C, nullptr, ld, cs->bound + J + nbo, cs->acc + J + nbo, kW, nc, mr,
                      1.f / (float)(1 << kVExp16), w.wp, kW, (int64_t)kW * nc, ws, f->status, s, &ws)) != CT_OK) {
    if (side) cudaStreamWaitEvent(s, la->ev_t, 0);
    return st;
  }
  // the next block's bounds: these columns' norms over rows J.. (kept by
  // the update below, which is orthogonal on those rows)
  if ((st = launch_norm_bound(cs->acc + J + nbo, nc, cs->bound + J + nbo, s)) != CT_OK) {
    if (side) cudaStreamWaitEvent(s, la->ev_t, 0);
    return st;
  }
  if (side) CT_CUDA_TRY(cudaStreamWaitEvent(s, la->ev_t, 0));
  {
    LaunchScope ls(K_TW, s, 2.0 * kW * kNB * nc * 1.5, 4.0 * kW * nc * (ws + 1));
    k_apply_tt16<kW><<<(unsigned)((nc + kTC - 1) / kTC), 256, kApplyTt16Smem, s>>>(
        w.wp, ws, (int64_t)kW * nc, kW, Ta, w.tab, Tb, nc, w.wh, w.wl, kW, w.winv);
    CT_LAUNCH_CHECK();
  }
  // C -= V W'  (K = 256)
  return tc_update16(w.vrh, w.vrl, kW, w.wh, w.wl, kW, w.winv, mr, nc, kW, C, ld, sms, f->status, s);
}

}  // namespace ctqr
