// qr_panel.cu -- FP64 panel factorization and its T factor.
//
// The panel is the mr x nbp block F[j0:m, j0:j0+nbp].  It is the GPU form of
// the paper's Compute_dense_QR task (Sec. II-C-3): annihilate everything
// below the diagonal with Householder reflectors, leave R on and above the
// diagonal and the reflectors below it, and produce the "S factor" needed to
// apply them as a block -- here the upper triangular T with
// H_0 H_1 ... H_{nbp-1} = I - V T V^T (Schreiber & Van Loan's compact WY form).
//
// One cooperative launch per panel.  CTA b holds rows [b*rp, (b+1)*rp) of the
// panel in shared memory (FP64) for the whole factorization, so the panel is
// read and written once.  Column k needs, from all rows:
//   sigma = sum_{r>k} a_rk^2,  alpha = a_kk,
//   d_c   = sum_{r>k} a_rk a_rc  and  a_kc          for c > k,
// which every CTA contributes as one partial vector; a single bounded grid
// barrier later, every CTA sums the vectors of all CTAs in the same fixed
// order (so all CTAs hold bitwise identical totals and the result does not
// depend on timing) and then, with
//   mu = sqrt(alpha^2 + sigma), beta = -sign(alpha) mu, tau = (beta-alpha)/beta,
//   v_r = a_rk/(alpha-beta)  (r > k), v_k = 1,
//   w_c = tau (a_kc + d_c/(alpha-beta)) = tau v^T a_c,
// updates its own rows: a_rc -= w_c v_r.  sigma == 0 gives tau = 0 (H = I),
// the same convention as LAPACK's dlarfg.
// After the last column each CTA adds its rows' share of the Gram matrix
// V^T V; the last CTA to finish sums the shares and builds T column by column:
//   T_ii = tau_i,  T[0:i, i] = -tau_i T[0:i, 0:i] (V^T V)[0:i, i].
#include <math.h>

#include "internal.cuh"

namespace ctqr {
namespace {

constexpr int kPT = 256;  // threads per CTA
constexpr int kNW = kPT / 32;
constexpr int kMaxNb = 64;

struct PanelArgs {
  void* P;               // &F[j0 + j0*ld]
  int64_t ld, mr;        // leading dimension, rows of the panel
  int nbp;               // columns of the panel (<= kMaxNb)
  int rp;                // rows per CTA
  int grid;              // CTAs
  double* tau;           // &tau[j0]
  double* T;             // nbp x nbp, leading dimension ldt
  int ldt;
  double* col_part;      // [2][grid][2*kMaxNb]
  double* gram_part;     // [grid][kMaxNb*(kMaxNb-1)/2]
  unsigned long long* bar;  // [0] grid-barrier counter, [1] finish counter
  int* status;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// S: storage type of the matrix; Mth: arithmetic of the panel's dot products
// and rank-1 updates (double for the FP64 factorization; float for the
// mixed-precision one, where sigma, alpha, beta, tau and T stay FP64).
template <typename S, typename Mth>
__global__ void __launch_bounds__(kPT, 1) k_panel(PanelArgs a) {
  extern __shared__ double smem[];
  double* red = smem;                               // [2*kMaxNb] reduced values
  double* wvd = red + 2 * kMaxNb;                   // [kMaxNb]  w_c
  double* scratch = wvd + kMaxNb;                   // [kNW][2*kMaxNb]
  Mth* wvm = (Mth*)(scratch + kNW * 2 * kMaxNb);    // [kMaxNb] w_c in the panel arithmetic
  Mth* slab = wvm + kMaxNb;                         // [nbp][rp], column-major
  __shared__ int s_last;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nbp = a.nbp, rp = a.rp;
  const int64_t rb = (int64_t)blockIdx.x * rp;      // first panel row of this CTA
  int64_t nr64 = a.mr - rb;
  const int nr = nr64 <= 0 ? 0 : (nr64 < rp ? (int)nr64 : rp);
  S* P = (S*)a.P;

  for (int c = 0; c < nbp; ++c)
    for (int r = tid; r < nr; r += kPT) slab[(size_t)c * rp + r] = (Mth)P[rb + r + c * a.ld];
  __syncthreads();

  for (int k = 0; k < nbp; ++k) {
    const int ne = nbp - k;                          // columns k..nbp-1
    const bool owner = (k >= rb) && (k < rb + nr);   // holds the diagonal row k
    const int kl = (int)(k - rb);                    // its local index when owner
    const int first = (int)(k + 1 - rb > 0 ? (k + 1 - rb < nr ? k + 1 - rb : nr) : 0);
    double* part = a.col_part + ((size_t)(k & 1) * a.grid + blockIdx.x) * (2 * kMaxNb);
    const Mth* colk = slab + (size_t)k * rp;
    // Partial vector: [q] = d_{k+q} (q = 0 is sigma, always accumulated in
    // FP64), [ne + q] = a_{k, k+q}.
    for (int q = warp; q < ne; q += kNW) {
      const Mth* colc = slab + (size_t)(k + q) * rp;
      double s = 0.0;
      if (q == 0) {
        for (int r = first + lane; r < nr; r += 32) s += (double)colk[r] * (double)colk[r];
      } else {
        Mth sm = (Mth)0;
        for (int r = first + lane; r < nr; r += 32) sm += colk[r] * colc[r];
        s = (double)sm;
      }
      s = warp_sum(s);
      if (lane == 0) {
        part[q] = s;
        part[ne + q] = owner ? (double)colc[kl] : 0.0;
      }
    }
    if (!grid_barrier(&a.bar[0], a.grid, a.status, kBarrierLimitNs)) return;

    // Deterministic reduction: thread t owns entry q = t % L of the partial
    // vectors (L = 2*ne) and sums the CTAs b = g, g+G, g+2G, ... of its group
    // g = t / L (G groups); the loads are independent and issued eight at a
    // time, then the G group sums are added in order.  Every CTA does the
    // same sums in the same order, so all hold identical totals.
    {
      const int L = 2 * ne;
      int groups = kPT / L;
      if (groups > kNW) groups = kNW;
      const int q = tid % L, grp = tid / L;
      const double* base = a.col_part + (size_t)(k & 1) * a.grid * (2 * kMaxNb);
      if (grp < groups) {
        double acc = 0.0;
        int b = grp;
        for (; b + 7 * groups < a.grid; b += 8 * groups) {
          double v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = __ldcg(base + (size_t)(b + u * groups) * (2 * kMaxNb) + q);
#pragma unroll
          for (int u = 0; u < 8; ++u) acc += v[u];
        }
        for (; b < a.grid; b += groups) acc += __ldcg(base + (size_t)b * (2 * kMaxNb) + q);
        scratch[grp * (2 * kMaxNb) + q] = acc;
      }
      __syncthreads();
      if (tid < L) {
        double s = 0.0;
        for (int w = 0; w < groups; ++w) s += scratch[w * (2 * kMaxNb) + tid];
        red[tid] = s;
      }
      __syncthreads();
    }

    const double sigma = red[0], alpha = red[ne];
    double beta = alpha, tau = 0.0, scale = 0.0;
    if (!isfinite(sigma) || !isfinite(alpha)) set_status(a.status, CT_ERR_NONFINITE);
    if (sigma != 0.0) {
      const double mu = sqrt(alpha * alpha + sigma);
      beta = alpha >= 0.0 ? -mu : mu;
      tau = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    if (tid > 0 && tid < ne) {
      wvd[tid] = tau * (red[ne + tid] + scale * red[tid]);
      wvm[tid] = (Mth)wvd[tid];  // converted once, not per row
    }
    __syncthreads();
    if (tau != 0.0) {
      const Mth sc = (Mth)scale;
      for (int r = first + tid; r < nr; r += kPT) {
        Mth* colr = slab + r;
        const Mth v = colr[(size_t)k * rp] * sc;
        colr[(size_t)k * rp] = v;
        for (int q = 1; q < ne; ++q) colr[(size_t)(k + q) * rp] -= wvm[q] * v;
      }
      if (owner && tid > 0 && tid < ne) slab[(size_t)(k + tid) * rp + kl] -= wvm[tid];
    }
    if (owner && tid == 0) slab[(size_t)k * rp + kl] = (Mth)beta;
    if (blockIdx.x == 0 && tid == 0) a.tau[k] = tau;
    __syncthreads();
  }

  // Write the factored rows back (storage precision).
  for (int c = 0; c < nbp; ++c)
    for (int r = tid; r < nr; r += kPT) P[rb + r + c * a.ld] = (S)slab[(size_t)c * rp + r];

  // This CTA's share of the strictly upper Gram matrix G = V^T V, packed as
  // p(i, j) = j(j-1)/2 + i for i < j (accumulated in the panel arithmetic).
  // v_i is 0 above row i and 1 on it.
  const int npairs = nbp * (nbp - 1) / 2;
  double* gp = a.gram_part + (size_t)blockIdx.x * (kMaxNb * (kMaxNb - 1) / 2);
  for (int j = 1 + warp; j < nbp; j += kNW) {
    for (int i = 0; i < j; ++i) {
      Mth sm = (Mth)0;
      for (int r = lane; r < nr; r += 32) {
        const int64_t gr = rb + r;
        if (gr < j) continue;  // v_j vanishes above its diagonal
        const Mth vj = gr == j ? (Mth)1 : slab[(size_t)j * rp + r];
        const Mth vi = gr == i ? (Mth)1 : (gr > i ? slab[(size_t)i * rp + r] : (Mth)0);
        sm += vi * vj;
      }
      const double s = warp_sum((double)sm);
      if (lane == 0) gp[j * (j - 1) / 2 + i] = s;
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned long long done = atomicAdd(&a.bar[1], 1ull);
    s_last = (done == (unsigned long long)(a.grid - 1));
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // Last CTA: total Gram (fixed CTA order) and T (FP64 either way).
  double* G = smem;                  // [npairs]
  double* Tm = G + npairs;           // [nbp][nbp] column-major
  double* tcol = Tm + nbp * nbp;     // [nbp]
  for (int p = tid; p < npairs; p += kPT) {
    double s = 0.0;
    for (int b = 0; b < a.grid; ++b) s += __ldcg(a.gram_part + (size_t)b * (kMaxNb * (kMaxNb - 1) / 2) + p);
    G[p] = s;
  }
  for (int p = tid; p < nbp * nbp; p += kPT) Tm[p] = 0.0;
  __syncthreads();
  for (int i = 0; i < nbp; ++i) {
    const double ti = __ldcg(a.tau + i);
    if (tid < i) {
      double s = 0.0;
      for (int b = tid; b < i; ++b) s += Tm[tid + b * nbp] * G[i * (i - 1) / 2 + b];
      tcol[tid] = -ti * s;
    }
    __syncthreads();
    if (tid < i) Tm[tid + i * nbp] = tcol[tid];
    if (tid == 0) Tm[i + i * nbp] = ti;
    __syncthreads();
  }
  for (int p = tid; p < nbp * nbp; p += kPT) {
    const int r = p % nbp, c = p / nbp;
    a.T[r + (size_t)c * a.ldt] = Tm[p];
  }
}

// CTAs for an mr-row panel: about 64 rows each, at most one per SM (measured:
// fewer, fuller CTAs were slower for both arithmetic types).
int panel_grid(int64_t mr, const DeviceInfo& di, size_t mth) {
  (void)mth;
  const int rows_per_cta = 64;
  int grid = (int)((mr + rows_per_cta - 1) / rows_per_cta);
  if (grid > di.sms) grid = di.sms;
  if (grid < 1) grid = 1;
  return grid;
}

size_t panel_smem_bytes(int nbp, int rp, size_t mth) {
  const size_t small = (size_t)(2 * kMaxNb + kMaxNb + kNW * 2 * kMaxNb) * sizeof(double) + kMaxNb * mth;
  size_t bytes = small + (size_t)nbp * rp * mth;
  const size_t t_need = ((size_t)nbp * (nbp - 1) / 2 + (size_t)nbp * nbp + nbp) * sizeof(double);
  return bytes < t_need ? t_need : bytes;
}

template <typename S, typename Mth>
ct_status launch_panel_t(ct_factor* f, int64_t j0, int nbp, double* T, cudaStream_t s,
                         const DeviceInfo& di) {
  const int64_t mr = f->m - j0;
  int grid = panel_grid(mr, di, sizeof(Mth));
  int rp = (int)((mr + grid - 1) / grid);
  const size_t smem = panel_smem_bytes(nbp, rp, sizeof(Mth));
  if (smem > (size_t)di.smem_optin) return CT_ERR_UNSUPPORTED;
  CT_CUDA_TRY(cudaFuncSetAttribute(k_panel<S, Mth>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_panel<S, Mth>, kPT, smem));
  if (per_sm < 1) return CT_ERR_UNSUPPORTED;
  if (grid > per_sm * di.sms) return CT_ERR_UNSUPPORTED;

  PanelArgs a;
  a.P = (char*)f->F + (size_t)(j0 + j0 * f->ld) * sizeof(S);
  a.ld = f->ld;
  a.mr = mr;
  a.nbp = nbp;
  a.rp = rp;
  a.grid = grid;
  a.tau = f->tau + j0;
  a.T = T;
  a.ldt = f->nb;
  a.col_part = f->partials;
  a.gram_part = f->partials + (size_t)2 * di.sms * 2 * kMaxNb;
  a.bar = f->barrier;
  a.status = f->status;
  CT_CUDA_TRY(cudaMemsetAsync(f->barrier, 0, 2 * sizeof(unsigned long long), s));
  void* args[] = {&a};
  LaunchScope ls(K_PANEL, s, 3.0 * (double)mr * nbp * nbp, 2.0 * (double)mr * nbp * sizeof(S));
  CT_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_panel<S, Mth>, dim3(grid), dim3(kPT), args, smem, s));
  return CT_OK;
}

}  // namespace

size_t panel_partials_elems(int sms, int nb) {
  (void)nb;
  return (size_t)2 * sms * 2 * kMaxNb + (size_t)sms * (kMaxNb * (kMaxNb - 1) / 2);
}

// Largest panel width <= want (halving when pow2) whose shared-memory slab
// fits for mr rows; mth = bytes of the panel arithmetic type.
int panel_width_that_fits(int64_t mr, int want, const DeviceInfo& di, size_t mth, bool pow2) {
  int grid = panel_grid(mr, di, mth);
  const int rp = (int)((mr + grid - 1) / grid);
  int nb = want > kMaxNb ? kMaxNb : want;
  while (nb > 8 && panel_smem_bytes(nb, rp, mth) > (size_t)di.smem_optin) nb = pow2 ? nb / 2 : nb - 8;
  return nb;
}

ct_status launch_panel(ct_factor* f, int64_t j0, int nbp, double* T, cudaStream_t s) {
  if (nbp < 1 || nbp > kMaxNb) return CT_ERR_INVALID;
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  return f->store == CT_F64 ? launch_panel_t<double, double>(f, j0, nbp, T, s, di)
                            : launch_panel_t<float, float>(f, j0, nbp, T, s, di);
}

}  // namespace ctqr
