// inner_update.cu -- one panel's block reflector applied to the rest of its
// 128-column outer block, C <- (I - V T V^T)^T C = C - V T^T V^T C, in one
// cooperative launch (the paper's Apply_left_Qt_of_dense_QR task, Sec.
// II-C-3, for the inner panels of the two-level factorization).
//
// The three-kernel form (V^T C split over rows, W' = T^T sum, C -= V W') costs
// three launches whose work is a few microseconds each; here every CTA owns
// a fixed range of rows of V and C, staged in shared memory in chunks of at
// most 320 rows (one chunk, kept between the phases, while the rows fit):
//   A. P_c = V^T C over the CTA's rows          (partial, to global)
//   -- grid barrier --
//   B. P = sum_c P_c, entries split over the CTAs, each summed over the
//      partials in a fixed order
//   -- grid barrier --
//   C. W' = T^T P (every CTA), then C -= V W' on the CTA's rows, chunk by
//      chunk (the last chunk first: it is still staged).
// FP32 arithmetic on the FP32-stored factor (T, kept in FP64, is rounded).
#include "internal.cuh"

namespace ctqr {
namespace {

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

template <int kIT>
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
  const int nchunk = (nrow + kIR - 1) / kIR;  // chunks of at most kIR rows
  const int c1 = (int)((mr + rows_per_cta - 1) / rows_per_cta);  // CTAs that own rows
  const int nc4 = (nc + 3) / 4;
  const int E = kIB * nc;  // entries of P, e = a * nc + c
  float* Cg = F + j0 + (j0 + nbp) * ld;  // C(r, c) at Cg[r + c * ld]
  // rows [lo, lo + n) of V and C (relative to j0) into shared memory
  auto load_chunk = [&](int64_t lo, int n) {
    __syncthreads();  // the previous chunk is no longer read
    for (int e = tid; e < n * kIB; e += kIT) {
      const int rr = e % n, a = e / n;
      const int64_t r = lo + rr;
      const bool v = a < nbp && r > a;  // unit lower: stored below the diagonal
      cp_async_f32(Vs + rr * kIV + a, v ? F + j0 + r + (j0 + a) * ld : F, v);
    }
    for (int e = tid; e < n * 4 * nc4; e += kIT) {
      const int rr = e % n, c = e / n;
      const bool v = c < nc;
      cp_async_f32(Cs + rr * kICS + c, v ? Cg + lo + rr + (int64_t)c * ld : F, v);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (tid < nbp && tid >= lo && tid < lo + n) Vs[(tid - lo) * kIV + tid] = 1.f;
    __syncthreads();
  };
  auto chunk_lo = [&](int q) { return r_lo + (int64_t)q * kIR; };
  auto chunk_n = [&](int q) { return (int)(r_hi - chunk_lo(q) < kIR ? r_hi - chunk_lo(q) : kIR); };
  // A. P_c(a, c) for a in [4 ag, 4 ag + 4), c in [4 cg, 4 cg + 4): thread
  // u = tid % 256 < 8 nc4 <= 192 of row group tid / 256 owns one such block
  // over the rows rr = group (mod groups) of all the CTA's chunks
  {
    constexpr int NG = kIT / 256;
    const int grp = tid / 256, u = tid % 256;
    const bool owner = u < (kIB / 4) * nc4;
    const int ag = u % (kIB / 4), cg = u / (kIB / 4);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int q = 0; q < nchunk; ++q) {
      const int n = chunk_n(q);
      load_chunk(chunk_lo(q), n);
      if (owner) {
        for (int rr = grp; rr < n; rr += NG) {
          const float4 v = *reinterpret_cast<const float4*>(Vs + rr * kIV + 4 * ag);
          const float4 c = *reinterpret_cast<const float4*>(Cs + rr * kICS + 4 * cg);
          const float vv[4] = {v.x, v.y, v.z, v.w}, cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(vv[i], cc[j], acc[i][j]);
        }
      }
    }
    if (NG > 1) {
      // the other groups' blocks through shared memory (Ps/Ws: free here)
      float* red = Ps;  // [NG - 1][192][16]
      __syncthreads();
      if (owner && grp > 0)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) red[((grp - 1) * 192 + u) * 16 + i * 4 + j] = acc[i][j];
      __syncthreads();
      if (owner && grp == 0)
        for (int g2 = 1; g2 < NG; ++g2)
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += red[((g2 - 1) * 192 + u) * 16 + i * 4 + j];
    }
    if (owner && grp == 0 && nrow > 0) {
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
  // C. C(r, c) -= sum_a V(r, a) W'(a, c) chunk by chunk, last chunk first
  // (it is still in shared memory), 4 x 4 tiles, results written back
  for (int q = nchunk - 1; q >= 0; --q) {
    const int64_t lo = chunk_lo(q);
    const int n = chunk_n(q);
    if (q != nchunk - 1) load_chunk(lo, n);
    const int rt = (n + 3) / 4;
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
        for (int i = 0; i < 4; ++i) vv[i] = r0 + i < n ? Vs[(r0 + i) * kIV + a] : 0.f;
        const float4 w = *reinterpret_cast<const float4*>(Ws + a * kICS + 4 * cg);
        const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(vv[i], ww[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (r0 + i < n)
#pragma unroll
          for (int j = 0; j < 4; ++j) Cs[(r0 + i) * kICS + 4 * cg + j] -= acc[i][j];
    }
    __syncthreads();
    for (int e = tid; e < n * nc; e += kIT) {
      const int rr = e % n, c = e / n;
      Cg[lo + rr + (int64_t)c * ld] = Cs[rr * kICS + c];
    }
  }
}

}  // namespace

ct_status inner_update_persist(ct_factor* f, int64_t j0, int nbp, int64_t cend, const double* Tp, double* work,
                               size_t work_elems, int sms, cudaStream_t s) {
  const int64_t nc = cend - j0 - nbp;
  if (f->store != CT_F32 || nbp < 1 || nbp > kIB || nc < 1 || nc > kINC || f->nb > kIB) return CT_ERR_UNSUPPORTED;
  const size_t smem = kInnerSmemFloats * sizeof(float);
  // 512 threads: two row groups in the V^T C phase, four warps per scheduler
  // to hide the shared-memory latencies of the update phase (136 ms against
  // 167 ms with 256 threads over the 256 x 256 system's factorization)
  constexpr int kIT = 512;
  const void* fn = (const void*)k_inner_update<kIT>;
  static bool attr = false;
  if (!attr) {
    CT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  int per_sm = 0;
  CT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kIT, smem));
  if (per_sm < 1) return CT_ERR_UNSUPPORTED;
  const int grid = sms;  // one CTA per SM (all co-resident for the grid barriers)
  const int64_t mr = f->m - j0;
  // rows beyond kIR per CTA are streamed in chunks of kIR (V and C read
  // twice, the second time mostly from L2)
  const int64_t rows = (mr + grid - 1) / grid;
  if (rows > INT32_MAX / 2) return CT_ERR_UNSUPPORTED;
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
  CT_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kIT), args, smem, s));
  return CT_OK;
}

}  // namespace ctqr
