// inner_update.cu -- one panel's block reflector applied to the rest of its
// 128-column outer block, C <- (I - V T V^T)^T C = C - V T^T V^T C, in one
// cooperative launch (the paper's Apply_left_Qt_of_dense_QR task, Sec.
// II-C-3, for the inner panels of the two-level factorization).
//
// The three-kernel form (V^T C split over rows, W' = T^T sum, C -= V W') costs
// three launches whose work is a few microseconds each; here every CTA owns
// a fixed range of rows of V and C, held in shared memory:
//   A. P_c = V^T C over the CTA's rows          (partial, to global)
//   -- grid barrier --
//   B. P = sum_c P_c, entries split over the CTAs, each summed over the
//      partials in a fixed order
//   -- grid barrier --
//   C. W' = T^T P (every CTA), then C -= V W' on the CTA's rows.
// FP32 arithmetic on the FP32-stored factor (T, kept in FP64, is rounded).
#include "internal.cuh"

namespace ctqr {
namespace {

constexpr int kIT = 256;    // threads
constexpr int kIB = 32;     // most reflectors (panel width)
constexpr int kIR = 320;    // most rows per CTA
constexpr int kINC = 96;    // most columns of C
constexpr int kIV = 36;     // row stride of V in shared memory (16-byte rows)
constexpr int kICS = 100;   // row stride of C, P and W' in shared memory
constexpr int kIT33 = 33;   // row stride of T
constexpr size_t kInnerSmemFloats =
    (size_t)kIR * kIV + (size_t)kIR * kICS + (size_t)kIB * kIT33 + (size_t)2 * kIB * kICS;

__device__ __forceinline__ float warp_sum_i(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kIT, 1) k_inner_update(float* __restrict__ F, int64_t ld, int64_t m, int64_t j0,
                                                         int nbp, int nc, const double* __restrict__ T, int ldt,
                                                         int rows_per_cta, float* __restrict__ part,
                                                         float* __restrict__ pred, unsigned long long* bar,
                                                         int* status) {
  extern __shared__ __align__(16) float si[];
  float* Vs = si;                    // V(rr, a) at rr * kIV + a (zero past nbp)
  float* Cs = Vs + kIR * kIV;        // C(rr, c) at rr * kICS + c
  float* Ts = Cs + kIR * kICS;       // T(b, a) at b * kIT33 + a
  float* Ps = Ts + kIB * kIT33;      // P(a, c) at a * kICS + c
  float* Ws = Ps + kIB * kICS;       // W'(a, c) at a * kICS + c
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int G = gridDim.x;
  const int64_t mr = m - j0;
  const int64_t r_lo = (int64_t)blockIdx.x * rows_per_cta;   // rows relative to j0
  const int64_t r_hi = r_lo + rows_per_cta < mr ? r_lo + rows_per_cta : mr;
  const int nrow = r_hi > r_lo ? (int)(r_hi - r_lo) : 0;
  const int c1 = (int)((mr + rows_per_cta - 1) / rows_per_cta);  // CTAs that own rows
  const int nc4 = (nc + 3) / 4;
  const int E = kIB * nc;  // entries of P, e = a * nc + c
  float* Cg = F + j0 + (j0 + nbp) * ld;  // C(r, c) at Cg[r + c * ld]
  if (nrow > 0) {
    for (int e = tid; e < nrow * kIB; e += kIT) {
      const int rr = e % nrow, a = e / nrow;
      const int64_t r = r_lo + rr;
      const bool v = a < nbp && r > a;  // unit lower: stored below the diagonal
      cp_async_f32(Vs + rr * kIV + a, v ? F + j0 + r + (j0 + a) * ld : F, v);
    }
    for (int e = tid; e < nrow * 4 * nc4; e += kIT) {
      const int rr = e % nrow, c = e / nrow;
      const bool v = c < nc;
      cp_async_f32(Cs + rr * kICS + c, v ? Cg + r_lo + rr + (int64_t)c * ld : F, v);
    }
    cp_async_commit();
    cp_async_wait_all();
  }
  __syncthreads();
  if (tid < nbp && tid >= r_lo && tid < r_hi) Vs[(tid - r_lo) * kIV + tid] = 1.f;
  __syncthreads();
  // A. P_c(a, c) for a in [4 ag, 4 ag + 4), c in [4 cg, 4 cg + 4)
  if (nrow > 0) {
    for (int t = tid; t < (kIB / 4) * nc4; t += kIT) {
      const int ag = t % (kIB / 4), cg = t / (kIB / 4);
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
      for (int rr = 0; rr < nrow; ++rr) {
        const float4 v = *reinterpret_cast<const float4*>(Vs + rr * kIV + 4 * ag);
        const float4 c = *reinterpret_cast<const float4*>(Cs + rr * kICS + 4 * cg);
        const float vv[4] = {v.x, v.y, v.z, v.w}, cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(vv[i], cc[j], acc[i][j]);
      }
      float* out = part + (size_t)blockIdx.x * E;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int a = 4 * ag + i, c = 4 * cg + j;
          if (c < nc) out[a * nc + c] = acc[i][j];
        }
    }
  }
  if (!grid_barrier(bar, (unsigned)G, status, kBarrierLimitNs)) return;
  // B. entries [e0, e1) of P over the partials of the CTAs that own rows
  {
    const int e0 = (int)((int64_t)blockIdx.x * E / G), e1 = (int)((int64_t)(blockIdx.x + 1) * E / G);
    for (int e = e0 + warp; e < e1; e += kIT / 32) {
      float s = 0.f;
      for (int z = lane; z < c1; z += 32) s += __ldcg(part + (size_t)z * E + e);
      s = warp_sum_i(s);
      if (lane == 0) pred[e] = s;
    }
  }
  if (!grid_barrier(bar, (unsigned)G, status, kBarrierLimitNs)) return;
  if (nrow == 0) return;
  for (int e = tid; e < kIB * 4 * nc4; e += kIT) {
    const int a = e / (4 * nc4), c = e % (4 * nc4);
    Ps[a * kICS + c] = c < nc ? __ldcg(pred + a * nc + c) : 0.f;
  }
  for (int e = tid; e < kIB * kIB; e += kIT) {
    const int b = e % kIB, a = e / kIB;
    Ts[b * kIT33 + a] = (a < nbp && b <= a) ? (float)T[b + (int64_t)a * ldt] : 0.f;
  }
  __syncthreads();
  // W'(a, c) = sum_{b <= a} T(b, a) P(b, c)
  for (int e = tid; e < kIB * 4 * nc4; e += kIT) {
    const int a = e / (4 * nc4), c = e % (4 * nc4);
    float w = 0.f;
    for (int b = 0; b <= a; ++b) w = fmaf(Ts[b * kIT33 + a], Ps[b * kICS + c], w);
    Ws[a * kICS + c] = w;
  }
  __syncthreads();
  // C. C(r, c) -= sum_a V(r, a) W'(a, c), 4 x 4 tiles, results into Cs
  {
    const int rt = (nrow + 3) / 4;
    for (int t = tid; t < rt * nc4; t += kIT) {
      const int cg = t % nc4, rg = t / nc4;  // lanes along columns: V reads are broadcasts
      float acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
      const int r0 = 4 * rg;
      for (int a = 0; a < kIB; ++a) {
        float vv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) vv[i] = r0 + i < nrow ? Vs[(r0 + i) * kIV + a] : 0.f;
        const float4 w = *reinterpret_cast<const float4*>(Ws + a * kICS + 4 * cg);
        const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(vv[i], ww[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (r0 + i < nrow)
#pragma unroll
          for (int j = 0; j < 4; ++j) Cs[(r0 + i) * kICS + 4 * cg + j] -= acc[i][j];
    }
  }
  __syncthreads();
  for (int e = tid; e < nrow * nc; e += kIT) {
    const int rr = e % nrow, c = e / nrow;
    Cg[r_lo + rr + (int64_t)c * ld] = Cs[rr * kICS + c];
  }
}

}  // namespace

ct_status inner_update_persist(ct_factor* f, int64_t j0, int nbp, int64_t cend, const double* Tp, double* work,
                               size_t work_elems, int sms, cudaStream_t s) {
  const int64_t nc = cend - j0 - nbp;
  if (f->store != CT_F32 || nbp < 1 || nbp > kIB || nc < 1 || nc > kINC || f->nb > kIB) return CT_ERR_UNSUPPORTED;
  const size_t smem = kInnerSmemFloats * sizeof(float);
  static bool attr = false;
  if (!attr) {
    CT_CUDA_TRY(cudaFuncSetAttribute(k_inner_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  int per_sm = 0;
  CT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_inner_update, kIT, smem));
  if (per_sm < 1) return CT_ERR_UNSUPPORTED;
  const int grid = sms;  // one CTA per SM (all co-resident for the grid barriers)
  const int64_t mr = f->m - j0;
  const int64_t rows = (mr + grid - 1) / grid;
  if (rows > kIR) return CT_ERR_UNSUPPORTED;
  const size_t E = (size_t)kIB * nc;
  if ((size_t)(grid + 1) * E * sizeof(float) > work_elems * sizeof(double)) return CT_ERR_UNSUPPORTED;
  float* part = (float*)work;
  float* pred = part + (size_t)grid * E;
  float* F = (float*)f->F;
  int64_t ld = f->ld, m = f->m, j0_ = j0;
  int nbp_ = nbp, nc_ = (int)nc, ldt = f->nb, rpc = (int)rows;
  const double* T = Tp;
  // the third barrier word: zeroed with the others before every panel launch,
  // and this launch follows the panel's on the same stream
  unsigned long long* bar = f->barrier + 2;
  int* status = f->status;
  void* args[] = {(void*)&F, (void*)&ld, (void*)&m, (void*)&j0_, (void*)&nbp_, (void*)&nc_, (void*)&T,
                  (void*)&ldt, (void*)&rpc, (void*)&part, (void*)&pred, (void*)&bar, (void*)&status};
  LaunchScope ls(K_INNER, s, 4.0 * (double)mr * nbp * nc, 2.0 * (double)mr * (nbp + nc) * 4.0);
  CT_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_inner_update, dim3(grid), dim3(kIT), args, smem, s));
  return CT_OK;
}

}  // namespace ctqr
