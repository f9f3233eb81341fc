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
#include <stdlib.h>

#include "internal.cuh"

namespace ctqr {
namespace {

constexpr int kPT = 256;  // threads per CTA
constexpr int kNW = kPT / 32;
constexpr int kMaxNb = 64;
// Bytes of the opt-in shared memory left for the panel kernels' static
// __shared__ variables (a few ints) when sizing their dynamic shared memory.
constexpr size_t kStaticSmemReserve = 1024;

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
  double* gram_part;     // [grid][kGramStride] partial Gram matrices, then the reduced one
  unsigned long long* bar;  // [0] grid-barrier counter, [1] finish counter
  int* status;
  int row0;              // rows held by CTA 0 (the panel's top nbp rows), the
                         // others rp each after them; 0: rp rows per CTA from row 0
  int dot2;              // Cholesky-QR: 1 = Gram and row solves as compensated
                         // FP32 products on an FP32 copy of the rows beside the
                         // FP64 one; 2 = the same with the FP32 rows only (tall
                         // panels whose FP64 rows do not fit); 0 = FP64
};

// First panel row and row count of CTA b.
__device__ __forceinline__ void cta_rows(const PanelArgs& a, int b, int64_t& rb, int& nr) {
  int64_t n64;
  if (a.row0 > 0) {
    rb = b == 0 ? 0 : a.row0 + (int64_t)(b - 1) * a.rp;
    const int cap = b == 0 ? a.row0 : a.rp;
    n64 = a.mr - rb;
    nr = n64 <= 0 ? 0 : (n64 < cap ? (int)n64 : cap);
  } else {
    rb = (int64_t)b * a.rp;
    n64 = a.mr - rb;
    nr = n64 <= 0 ? 0 : (n64 < a.rp ? (int)n64 : a.rp);
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Householder factorization of the panel whose rows this CTA holds in `slab`
// (column-major, rp rows per column, already loaded), write-back of V / R in
// the storage type, tau, and T by the last CTA to finish.  `small` holds the
// reduction buffers (kSmallDoubles doubles plus kMaxNb Mth values);
// `smem` is the start of the CTA's shared memory, reused for T at the end.
// S: storage type of the matrix; Mth: arithmetic of the panel's dot products
// and rank-1 updates (double for the FP64 factorization; float for the
// mixed-precision one, where sigma, alpha, beta, tau and T stay FP64).
constexpr int kSmallDoubles = 2 * kMaxNb + kMaxNb + kNW * 2 * kMaxNb;

template <typename S, typename Mth>
__device__ void panel_householder(const PanelArgs& a, Mth* slab, double* small, double* smem) {
  double* red = small;                              // [2*kMaxNb] reduced values
  double* wvd = red + 2 * kMaxNb;                   // [kMaxNb]  w_c
  double* scratch = wvd + kMaxNb;                   // [kNW][2*kMaxNb]
  Mth* wvm = (Mth*)(scratch + kNW * 2 * kMaxNb);    // [kMaxNb] w_c in the panel arithmetic
  __shared__ int s_last;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nbp = a.nbp, rp = a.rp;
  int64_t rb;                                       // first panel row of this CTA
  int nr;
  cta_rows(a, blockIdx.x, rb, nr);
  S* P = (S*)a.P;
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


template <typename S, typename Mth>
__global__ void __launch_bounds__(kPT, 1) k_panel(PanelArgs a) {
  extern __shared__ double smem[];
  double* small = smem;
  Mth* slab = (Mth*)(small + kSmallDoubles) + kMaxNb;  // after the kMaxNb Mth values of w
  const int tid = threadIdx.x;
  int64_t rb;
  int nr;
  cta_rows(a, blockIdx.x, rb, nr);
  const S* P = (const S*)a.P;
  for (int c = 0; c < a.nbp; ++c)
    for (int r = tid; r < nr; r += kPT) slab[(size_t)c * a.rp + r] = (Mth)P[rb + r + c * a.ld];
  __syncthreads();
  panel_householder<S, Mth>(a, slab, small, smem);
}

// ---------------------------------------------------------------------------
// Cholesky-QR panel with Householder reconstruction (FP32-stored factors).
//
// The per-column Householder panel above needs one grid barrier per column.
// For a full-rank, reasonably conditioned panel P (mr x nbp) the same
// Householder factorization can be reached with two:
//   1. G = P^T P (FP64; every CTA its rows, then a split reduction) and its
//      Cholesky factor G = R1^T R1, so Q = P R1^{-1} has orthonormal columns;
//   2. the "modified LU" of Ballard et al. (Reconstructing Householder vectors
//      from tall-skinny QR, 2015): Q - [S; 0] = L U without pivoting, the sign
//      s_i = -sign of the current diagonal entry, so every pivot has modulus
//      >= 1.  Then V = L (unit lower trapezoidal), T = -U S L1^{-T} (upper),
//      I - V T V^T has Q S as its first nbp columns and the panel's R is S R1.
// Only the top nbp rows of Q are formed explicitly (every CTA does the small
// nbp x nbp algebra redundantly, in the same order, so all agree bitwise); the
// rows below are V2 = Q2 U^{-1} = P2 M^{-1} with M = U R1, one triangular
// solve per row.  tau_i = T_ii and V^T V are those of the equivalent sequence
// of reflectors, so the 128-column outer update's S = T^{-1} form applies
// unchanged.  When the Cholesky factor breaks down or kappa_1(R1) exceeds
// kCqrMaxCond (so Q would be orthonormal only to kappa^2 u), every CTA falls
// back to the per-column Householder path on the same resident slab.
constexpr double kCqrMaxCond = 3.0e3;
constexpr int kGramStride = kMaxNb * (kMaxNb + 1) / 2;  // doubles per CTA partial Gram

__device__ __forceinline__ void tri_index(int e, int& i, int& j) {
  // e = j (j + 1) / 2 + i, 0 <= i <= j
  int jj = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (jj * (jj + 1) / 2 > e) --jj;
  while ((jj + 1) * (jj + 2) / 2 <= e) ++jj;
  j = jj;
  i = e - jj * (jj + 1) / 2;
}

__host__ __device__ inline int pow2_at_least(int n) {
  int p = 1;
  while (p < n) p *= 2;
  return p;
}

// X = A^{-1} for the upper triangular n x n matrix a(i, j) (i <= j), in P x P
// shared storage with leading dimension P (P a power of two >= n; rows and
// columns >= n act as the identity).  Block doubling: the diagonal
// reciprocals, then for s = 1, 2, 4, ... and every pair of diagonal blocks
// A = [p, p+s), C = [p+s, p+2s): X_AC = -X_A (a_AC X_C).  Each step is a pair
// of small products spread over all threads (no long serial chains, which
// GB300's FP64 pipe makes expensive).  tmp: P x P scratch.
template <typename Acc>
__device__ void tri_inv_upper(Acc a, double* X, double* tmp, int n, int P) {
  const int tid = threadIdx.x;
  for (int e = tid; e < P * P; e += kPT) {
    const int i = e % P, j = e / P;
    X[e] = i == j ? (i < n ? 1.0 / a(i, i) : 1.0) : 0.0;
  }
  __syncthreads();
  for (int s = 1; s < P; s *= 2) {
    const int ent = (P / (2 * s)) * s * s;
    for (int e = tid; e < ent; e += kPT) {
      const int pr = e / (s * s), rr = e % (s * s), r = rr % s, c = rr / s;
      const int p0 = pr * 2 * s, gi = p0 + r, gc = p0 + s + c;
      double acc = 0.0;
      for (int k = 0; k <= c; ++k) {  // X_C is upper triangular
        const int gk = p0 + s + k;
        if (gi < n && gk < n) acc += a(gi, gk) * X[gk + gc * P];
      }
      tmp[gi + gc * P] = acc;
    }
    __syncthreads();
    for (int e = tid; e < ent; e += kPT) {
      const int pr = e / (s * s), rr = e % (s * s), r = rr % s, c = rr / s;
      const int p0 = pr * 2 * s, gi = p0 + r, gc = p0 + s + c;
      double acc = 0.0;
      for (int k = r; k < s; ++k) acc += X[gi + (p0 + k) * P] * tmp[(p0 + k) + gc * P];  // X_A upper
      X[gi + gc * P] = -acc;
    }
    __syncthreads();
  }
}

// 1/sqrt(d) and 1/x in FP64 from an FP32 seed refined by two Newton-Raphson
// steps (y <- y (3 - d y^2) / 2 and y <- y (2 - x y)); the seed's relative
// error ~1e-7 squares at every step, so the result is within a few FP64 ulps.
// A few FP64 instructions instead of a full-precision square root or
// division: on GB300 every FP64 instruction of a single thread costs the
// FP64 pipe the time of a whole warp.  Outside the FP32 range the exact
// operations are used.
__device__ __forceinline__ double rsqrt_nr(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf((float)d);
  y = y * (1.5 - 0.5 * d * y * y);
  y = y * (1.5 - 0.5 * d * y * y);
  return y;
}

__device__ __forceinline__ double rcp_nr(double x) {
  const double ax = fabs(x);
  if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
  double y = (double)(1.0f / (float)x);
  y = y * (2.0 - x * y);
  y = y * (2.0 - x * y);
  return y;
}

// Compensated dot product on the FP32 pipes: Dot2 of Ogita, Rump and Oishi
// (2005), built from the error-free transformations TwoProduct (by FMA) and
// TwoSum (Knuth).  s + c carries the sum of products with about twice FP32's
// precision; every operation is an explicitly rounded intrinsic so the
// compiler cannot contract the transformations.  On GB300 this costs ten
// FP32 instructions per term against one FP64 FMA, and the FP32 pipes issue
// 64 times as many lanes per clock.
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x, float y) {
    const float p = __fmul_rn(x, y);
    const float pe = __fmaf_rn(x, y, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(pe, e));
  }
  // a term far below s (the low part of a split factor): into c directly
  __device__ __forceinline__ void add_small(float x, float y) { c = __fmaf_rn(x, y, c); }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <typename S>
__global__ void __launch_bounds__(kPT, 1) k_panel_cqr(PanelArgs a) {
  extern __shared__ double smem[];
  const int nbp = a.nbp, rp = a.rp, tid = threadIdx.x;
  const int P = pow2_at_least(nbp);           // leading dimension of the small matrices
  const int nn = P * P;
  // with a.dot2: the rows in FP32 (exact: the data is FP32) and M^{-1} split
  // into FP32 high and low parts; with a.dot2 == 2 only the FP32 rows are
  // kept (they come first, the FP64 small matrices after them)
  const bool dot2 = a.dot2 != 0, f32only = a.dot2 == 2;
  double* slab = f32only ? nullptr : smem;    // [nbp][rp] this CTA's rows (FP64)
  double* G = f32only ? (double*)((char*)smem + (((size_t)nbp * rp * sizeof(float) + 15) & ~(size_t)15))
                      : slab + (size_t)nbp * rp;  // Gram, then R1 in its upper part
  double* Ri = G + nn;                        // R1^{-1} (upper), later T
  double* W = Ri + nn;                        // P1, then Q1 - S -> L1 (strict lower) / U (upper)
  double* M = W + nn;                         // scratch, then M^{-1} = R1^{-1} U^{-1}
  double* X = M + nn;                         // scratch / U^{-1} / (L1^T)^{-1}
  double* sv = X + nn;                        // [P] s_i
  double* dv = sv + P;                        // [P] column sums
  float* slabf = f32only ? (float*)smem : (float*)(dv + P);  // [nbp][rp]
  float* Mh = f32only ? (float*)(dv + P) : slabf + (size_t)nbp * rp;
  float* Ml = Mh + nn;
  __shared__ int s_ok;
  int64_t rb;
  int nr;
  cta_rows(a, blockIdx.x, rb, nr);
  S* P_ = (S*)a.P;

  // the slab, eight columns' loads in flight per thread
  for (int r = tid; r < nr; r += kPT) {
    const S* src = P_ + rb + r;
    int c = 0;
    for (; c + 8 <= nbp; c += 8) {
      S v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = src[(int64_t)(c + u) * a.ld];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (!f32only) slab[(size_t)(c + u) * rp + r] = (double)v[u];
        if (dot2) slabf[(size_t)(c + u) * rp + r] = (float)v[u];
      }
    }
    for (; c < nbp; ++c) {
      const S v = src[(int64_t)c * a.ld];
      if (!f32only) slab[(size_t)c * rp + r] = (double)v;
      if (dot2) slabf[(size_t)c * rp + r] = (float)v;
    }
  }
  // the top nbp rows of the panel (held by CTA 0, read by all before CTA 0
  // can overwrite them, i.e. before the second barrier)
  for (int e = tid; e < nbp * nbp; e += kPT) {
    const int r = e % nbp, c = e / nbp;
    W[r + c * P] = (double)P_[r + (int64_t)c * a.ld];
  }
  __syncthreads();

  // 1. This CTA's share of the upper Gram matrix, packed.
  const int ng = nbp * (nbp + 1) / 2;
  double* gp = a.gram_part + (size_t)blockIdx.x * kGramStride;
  // whole rounds of kPT entries, one thread per entry; the remaining entries
  // (if few) with g threads per entry over interleaved rows, so that no
  // round runs on a handful of threads
  const int full = (ng / kPT) * kPT, rem = ng - full;
  int g = 1;
  while (rem > 0 && g < 32 && rem * g * 2 <= kPT) g *= 2;
  const int split_from = g > 1 ? full : ng;
  for (int e = tid; e < split_from; e += kPT) {
    int i, j;
    tri_index(e, i, j);
    if (dot2) {
      const float* ci = slabf + (size_t)i * rp;
      const float* cj = slabf + (size_t)j * rp;
      Dot2 d0, d1;
      int r = 0;
      for (; r + 1 < nr; r += 2) {
        d0.add(ci[r], cj[r]);
        d1.add(ci[r + 1], cj[r + 1]);
      }
      if (r < nr) d0.add(ci[r], cj[r]);
      gp[e] = d0.value() + d1.value();
    } else {
      const double* ci = slab + (size_t)i * rp;
      const double* cj = slab + (size_t)j * rp;
      double s0 = 0.0, s1 = 0.0;
      int r = 0;
      for (; r + 1 < nr; r += 2) {
        s0 += ci[r] * cj[r];
        s1 += ci[r + 1] * cj[r + 1];
      }
      if (r < nr) s0 += ci[r] * cj[r];
      gp[e] = s0 + s1;
    }
  }
  // rem * g <= kPT; g is a power of two <= 32, so the groups of g lanes never
  // straddle a warp; whole warps take part in the shuffles
  if (g > 1 && tid < (rem * g + 31) / 32 * 32) {
    const bool act = tid < rem * g;
    const int e = full + tid / g, part = tid % g;
    double s = 0.0;
    if (act) {
      int i, j;
      tri_index(e, i, j);
      if (dot2) {
        const float* ci = slabf + (size_t)i * rp;
        const float* cj = slabf + (size_t)j * rp;
        Dot2 d;
        for (int r = part; r < nr; r += g) d.add(ci[r], cj[r]);
        s = d.value();
      } else {
        const double* ci = slab + (size_t)i * rp;
        const double* cj = slab + (size_t)j * rp;
        for (int r = part; r < nr; r += g) s += ci[r] * cj[r];
      }
    }
    for (int o = g / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, g);
    if (act && part == 0) gp[e] = s;
  }
  if (!grid_barrier(&a.bar[0], a.grid, a.status, kBarrierLimitNs)) return;
  // Split reduction: CTA c sums entries [c ng / grid, (c+1) ng / grid) over
  // all CTAs' partials in a fixed order.
  double* gred = a.gram_part + (size_t)a.grid * kGramStride;
  {
    const int e0 = (int)((int64_t)blockIdx.x * ng / a.grid), e1 = (int)((int64_t)(blockIdx.x + 1) * ng / a.grid);
    const int lane = tid & 31, warp = tid >> 5;
    for (int e = e0 + warp; e < e1; e += kNW) {
      double s = 0.0;
      for (int b = lane; b < a.grid; b += 32) s += __ldcg(a.gram_part + (size_t)b * kGramStride + e);
      s = warp_sum(s);
      if (lane == 0) gred[e] = s;
    }
  }
  if (!grid_barrier(&a.bar[0], a.grid, a.status, kBarrierLimitNs)) return;

  // 2. Every CTA: the full Gram matrix (identity outside nbp), its Cholesky
  //    factor R1 (upper, in G; one reciprocal per pivot).
  for (int e = tid; e < nn; e += kPT) {
    const int i = e % P, j = e / P;
    G[e] = (i >= nbp || j >= nbp) ? (i == j ? 1.0 : 0.0) : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < ng; e += kPT) {
    int i, j;
    tri_index(e, i, j);
    const double v = __ldcg(gred + e);
    G[i + j * P] = v;
    G[j + i * P] = v;
  }
  if (tid == 0) s_ok = 1;
  __syncthreads();
  for (int k = 0; k < nbp; ++k) {
    if (tid == 0) {
      const double d = G[k + k * P];
      if (!(d > 0.0) || !isfinite(d)) s_ok = 0;
      const double y = s_ok ? rsqrt_nr(d) : 1.0;  // 1 / sqrt(d)
      G[k + k * P] = s_ok ? d * y : 1.0;
      dv[0] = y;
    }
    __syncthreads();
    const double rinv = dv[0];
    for (int j = k + 1 + tid; j < nbp; j += kPT) G[k + j * P] *= rinv;
    __syncthreads();
    const int w = nbp - k - 1;  // trailing block (k+1..nbp-1)^2, upper part
    for (int e = tid; e < w * w; e += kPT) {
      const int i = k + 1 + e % w, j = k + 1 + e / w;
      if (i <= j) G[i + j * P] -= G[k + i * P] * G[k + j * P];
    }
    __syncthreads();
  }
  // R1^{-1} and kappa_1(R1) = ||R1||_1 ||R1^{-1}||_1
  tri_inv_upper(
      [&](int i, int j) { return G[i + j * P]; }, Ri, M, nbp, P);
  // (an estimate: FP32 sums of the FP64 entries suffice)
  if (tid < 32) {
    float n1 = 0.f, n2 = 0.f;
    for (int j = tid; j < nbp; j += 32) {
      float s1 = 0.f, s2 = 0.f;
      for (int i = 0; i <= j; ++i) {
        s1 += fabsf((float)G[i + j * P]);
        s2 += fabsf((float)Ri[i + j * P]);
      }
      n1 = fmaxf(n1, s1);
      n2 = fmaxf(n2, s2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n1 = fmaxf(n1, __shfl_xor_sync(0xffffffffu, n1, o));
      n2 = fmaxf(n2, __shfl_xor_sync(0xffffffffu, n2, o));
    }
    if (tid == 0 && !(n1 * n2 <= (float)kCqrMaxCond)) s_ok = 0;
  }
  __syncthreads();
  if (!s_ok) {
    // per-column Householder on the same slab; G.. onward is free (FP32
    // rows only: the per-column panel in FP32 arithmetic on them)
    if (f32only) panel_householder<S, float>(a, slabf, G, smem);
    else panel_householder<S, double>(a, slab, G, smem);
    return;
  }

  // 3. Q1 = P1 R1^{-1} (into M, then W), then the modified LU of Q1 - S in
  //    place (one reciprocal per pivot).
  for (int e = tid; e < nbp * nbp; e += kPT) {
    const int r = e % nbp, j = e / nbp;
    double s = 0.0;
    for (int k = 0; k <= j; ++k) s += W[r + k * P] * Ri[k + j * P];
    M[r + j * P] = s;
  }
  __syncthreads();
  for (int e = tid; e < nbp * nbp; e += kPT) {
    const int r = e % nbp, j = e / nbp;
    W[r + j * P] = M[r + j * P];
  }
  __syncthreads();
  for (int i = 0; i < nbp; ++i) {
    if (tid == 0) {
      const double q = W[i + i * P];
      const double si = q >= 0.0 ? -1.0 : 1.0;
      sv[i] = si;
      W[i + i * P] = q - si;  // |pivot| >= 1
      dv[0] = rcp_nr(q - si);
    }
    __syncthreads();
    const double pinv = dv[0];
    for (int r = i + 1 + tid; r < nbp; r += kPT) W[r + i * P] *= pinv;
    __syncthreads();
    const int w = nbp - i - 1;
    for (int e = tid; e < w * w; e += kPT) {
      const int r = i + 1 + e % w, c = i + 1 + e / w;
      W[r + c * P] -= W[r + i * P] * W[i + c * P];
    }
    __syncthreads();
  }
  // U^{-1} (into X), then M^{-1} = (U R1)^{-1} = R1^{-1} U^{-1} (into M)
  tri_inv_upper(
      [&](int i, int j) { return W[i + j * P]; }, X, M, nbp, P);
  for (int e = tid; e < nbp * nbp; e += kPT) {
    const int i = e % nbp, j = e / nbp;
    double s = 0.0;
    if (i <= j)
      for (int k = i; k <= j; ++k) s += Ri[i + k * P] * X[k + j * P];
    M[i + j * P] = s;
  }
  __syncthreads();
  if (dot2) {
    for (int e = tid; e < nn; e += kPT) {
      const double mv = M[e];
      const float h = (float)mv;
      Mh[e] = h;
      Ml[e] = (float)(mv - (double)h);
    }
    __syncthreads();
  }

  // 4. This CTA's rows: V2 = P2 M^{-1} (rows with panel index >= nbp, columns
  //    from the last so that each row is updated in place); the top nbp rows
  //    (CTA 0) become R = S R1 on/above and L1 below the diagonal.
  for (int r = tid; r < nr; r += kPT) {
    const int64_t gr = rb + r;
    if (gr >= nbp) {
      // FP32 result (the factor's storage type) of a compensated product
      // with the split M^{-1}; the inputs are the unmodified FP32 copy
      if (dot2) {
        for (int j = nbp - 1; j >= 0; --j) {
          Dot2 d;
          for (int i = 0; i <= j; ++i) {
            const float x = slabf[(size_t)i * rp + r];
            d.add(x, Mh[i + j * P]);
            d.add_small(x, Ml[i + j * P]);
          }
          const float y = __fadd_rn(d.s, d.c);
          if (f32only) slabf[(size_t)j * rp + r] = y;  // column j read above, before this write
          else slab[(size_t)j * rp + r] = (double)y;
        }
      } else {
        for (int j = nbp - 1; j >= 0; --j) {
          double acc = 0.0;
          for (int i = 0; i <= j; ++i) acc += slab[(size_t)i * rp + r] * M[i + j * P];
          slab[(size_t)j * rp + r] = acc;
        }
      }
    } else {
      const int i = (int)gr;
      for (int j = 0; j < nbp; ++j) {
        const double y = j >= i ? sv[i] * G[i + j * P] : W[i + j * P];
        if (f32only) slabf[(size_t)j * rp + r] = (float)y;
        else slab[(size_t)j * rp + r] = y;
      }
    }
  }
  __syncthreads();
  for (int c = 0; c < nbp; ++c)
    for (int r = tid; r < nr; r += kPT)
      P_[rb + r + c * a.ld] = f32only ? (S)slabf[(size_t)c * rp + r] : (S)slab[(size_t)c * rp + r];

  // 5. CTA 0 (which holds only the top rows, so it has no row solves):
  //    T = -U S L1^{-T} and tau = diag(T).  L1^{-T} is the inverse of the
  //    unit upper triangular L1^T.
  if (blockIdx.x != 0) return;
  tri_inv_upper(
      [&](int i, int j) { return i == j ? 1.0 : W[j + i * P]; }, X, M, nbp, P);
  for (int e = tid; e < nbp * nbp; e += kPT) {
    const int i = e % nbp, j = e / nbp;
    double s = 0.0;
    if (i <= j)
      for (int k = i; k <= j; ++k) s += W[i + k * P] * sv[k] * X[k + j * P];
    Ri[i + j * P] = i <= j ? -s : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < nbp * nbp; e += kPT) {
    const int i = e % nbp, j = e / nbp;
    a.T[i + (size_t)j * a.ldt] = Ri[i + j * P];
  }
  for (int i = tid; i < nbp; i += kPT) a.tau[i] = Ri[i + i * P];
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

// dot2: 0 FP64 rows, 1 FP64 and FP32 rows, 2 FP32 rows only.
size_t panel_cqr_smem_bytes(int nbp, int rp, int dot2) {
  const size_t P = (size_t)pow2_at_least(nbp);
  const size_t rows64 = dot2 == 2 ? 0 : (size_t)nbp * rp * sizeof(double);
  const size_t rows32 = dot2 == 0 ? 0 : (((size_t)nbp * rp * sizeof(float) + 15) & ~(size_t)15);
  size_t bytes = rows64 + rows32 + (5 * P * P + 2 * P) * sizeof(double) +
                 (dot2 ? 2 * P * P * sizeof(float) : 0);  // split M^{-1}
  // the Householder fallback: its buffers in place of G.., T at the start
  const size_t fb = rows64 + rows32 + (kSmallDoubles + kMaxNb) * sizeof(double);
  const size_t t_need = ((size_t)nbp * (nbp - 1) / 2 + (size_t)nbp * nbp + nbp) * sizeof(double);
  bytes = bytes < fb ? fb : bytes;
  return bytes < t_need ? t_need : bytes;
}

size_t panel_smem_bytes(int nbp, int rp, size_t mth) {
  const size_t small = (size_t)(2 * kMaxNb + kMaxNb + kNW * 2 * kMaxNb) * sizeof(double) + kMaxNb * mth;
  size_t bytes = small + (size_t)nbp * rp * mth;
  const size_t t_need = ((size_t)nbp * (nbp - 1) / 2 + (size_t)nbp * nbp + nbp) * sizeof(double);
  return bytes < t_need ? t_need : bytes;
}

// Cholesky-QR panels are used for FP32-stored factors unless
// CTQR_PANEL_HOUSEHOLDER=1 asks for the per-column kernel everywhere.
bool cqr_enabled() {
  static const bool on = [] {
    const char* e = getenv("CTQR_PANEL_HOUSEHOLDER");
    return !(e && *e == '1');
  }();
  return on;
}

template <typename S, typename Mth>
ct_status launch_panel_t(ct_factor* f, int64_t j0, int nbp, double* T, cudaStream_t s,
                         const DeviceInfo& di) {
  const int64_t mr = f->m - j0;
  int grid = panel_grid(mr, di, sizeof(Mth));
  if (f->panel_cap > 0 && grid > f->panel_cap) grid = f->panel_cap;
  int rp = (int)((mr + grid - 1) / grid);
  // dynamic shared memory may use the opt-in limit minus the kernels' few
  // bytes of static shared memory
  const size_t limit = (size_t)di.smem_optin - kStaticSmemReserve;
  // Cholesky-QR: CTA 0 holds only the top nbp rows (it forms T while the
  // others solve their rows), the other CTAs the rest in equal parts
  int row0 = 0, rp_c = rp;
  if (grid >= 2 && mr > nbp) {
    rp_c = (int)((mr - nbp + grid - 2) / (grid - 1));
    if (rp_c < nbp) rp_c = nbp;
  }
  const bool cqr_ok = sizeof(S) == 4 && cqr_enabled() && rp >= nbp;
  // compensated FP32 Gram and row solves beside the FP64 rows when both fit;
  // for taller panels the FP32 rows alone (compensated products throughout)
  int dot2 = 0;
  bool cqr = false;
  if (cqr_ok && panel_cqr_smem_bytes(nbp, rp_c, 0) <= limit) {
    cqr = true;
    dot2 = panel_cqr_smem_bytes(nbp, rp_c, 1) <= limit ? 1 : 0;
  } else if (cqr_ok && panel_cqr_smem_bytes(nbp, rp_c, 2) <= limit) {
    cqr = true;
    dot2 = 2;
  }
  if (cqr) {
    if (grid >= 2 && mr > nbp) row0 = nbp;
    rp = rp_c;
  }
  const void* fn = cqr ? (const void*)k_panel_cqr<S> : (const void*)k_panel<S, Mth>;
  const size_t smem = cqr ? panel_cqr_smem_bytes(nbp, rp, dot2) : panel_smem_bytes(nbp, rp, sizeof(Mth));
  if (smem > limit) return CT_ERR_UNSUPPORTED;
  CT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPT, smem));
  if (per_sm < 1) return CT_ERR_UNSUPPORTED;
  if (grid > per_sm * di.sms) return CT_ERR_UNSUPPORTED;

  PanelArgs a;
  a.P = (char*)f->F + (size_t)(j0 + j0 * f->ld) * sizeof(S);
  a.ld = f->ld;
  a.mr = mr;
  a.nbp = nbp;
  a.rp = rp;
  a.grid = grid;
  a.row0 = row0;
  a.dot2 = dot2;
  a.tau = f->tau + j0;
  a.T = T;
  a.ldt = f->nb;
  a.col_part = f->partials;
  a.gram_part = f->partials + (size_t)2 * (di.sms + 1) * 2 * kMaxNb;
  a.bar = f->barrier;
  a.status = f->status;
  // the panel's two words and the third, used by the inner update that follows
  CT_CUDA_TRY(cudaMemsetAsync(f->barrier, 0, 3 * sizeof(unsigned long long), s));
  void* args[] = {&a};
  LaunchScope ls(K_PANEL, s, 3.0 * (double)mr * nbp * nbp, 2.0 * (double)mr * nbp * sizeof(S));
  CT_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kPT), args, smem, s));
  return CT_OK;
}

}  // namespace

size_t panel_partials_elems(int sms, int nb) {
  (void)nb;
  // column partials [2][sms + 1][2*kMaxNb]; per-CTA Gram partials for up to
  // sms + 1 CTAs and the reduced Gram of the Cholesky-QR panel after them
  return (size_t)2 * (sms + 1) * 2 * kMaxNb + (size_t)(sms + 2) * kGramStride;
}

// Largest panel width <= want (halving when pow2) whose shared-memory slab
// fits for mr rows; mth = bytes of the panel arithmetic type.
int panel_width_that_fits(int64_t mr, int want, const DeviceInfo& di, size_t mth, bool pow2) {
  int grid = panel_grid(mr, di, mth);
  const int rp = (int)((mr + grid - 1) / grid);
  int nb = want > kMaxNb ? kMaxNb : want;
  while (nb > 8 && panel_smem_bytes(nb, rp, mth) > (size_t)di.smem_optin - kStaticSmemReserve)
    nb = pow2 ? nb / 2 : nb - 8;
  return nb;
}

bool panel_fits_ctas(int64_t mr, int nbp, int ctas, const DeviceInfo& di) {
  if (ctas < 1) return false;
  const int rp = (int)((mr + ctas - 1) / ctas);
  return panel_smem_bytes(nbp, rp, sizeof(float)) <= (size_t)di.smem_optin - kStaticSmemReserve;
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
