// internal.cuh -- declarations shared by the translation units of libctqr.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ctqr.h"

namespace ctqr {

// ---------------------------------------------------------------------------
// Errors.  Host code returns ct_status; device code records the first error in
// a status word (int) in device memory with atomicCAS(status, 0, code).
// ---------------------------------------------------------------------------
#define CT_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t e__ = (expr);                               \
    if (e__ != cudaSuccess) {                               \
      ctqr::note_cuda_error(e__, #expr, __FILE__, __LINE__); \
      return e__ == cudaErrorMemoryAllocation ? CT_ERR_NOMEM : CT_ERR_CUDA; \
    }                                                       \
  } while (0)

#define CT_LAUNCH_CHECK() CT_CUDA_TRY(cudaGetLastError())

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Device-side failure recording (first error wins).
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *(const volatile int*)p;
}

// Bounded grid-wide barrier for kernels launched cooperatively (all CTAs
// co-resident).  `counter` is a 64-bit arrival counter zeroed before the
// launch; the barrier round r completes when the counter reaches
// (r+1)*nblocks.  Each waiting CTA spins at most `limit_ns` nanoseconds; on
// timeout it records CT_ERR_TIMEOUT and returns false, and a CTA that sees
// another CTA's error also returns false, so every CTA leaves in bounded time.
__device__ __forceinline__ bool grid_barrier(unsigned long long* counter, unsigned nblocks,
                                             int* status, uint64_t limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    unsigned long long arrival = atomicAdd(counter, 1ull);
    unsigned long long target = (arrival / nblocks + 1ull) * nblocks;
    uint64_t t0 = globaltimer_ns();
    while (ld_acquire_u64(counter) < target) {
      if (ld_volatile_i32(status) != 0) { ok = 0; break; }
      if (globaltimer_ns() - t0 > limit_ns) { set_status(status, CT_ERR_TIMEOUT); ok = 0; break; }
      __nanosleep(20);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

constexpr uint64_t kBarrierLimitNs = 2000000000ull;  // 2 s per wait

// 4-byte asynchronous copy global -> shared; an invalid element is filled
// with zero (source size 0: nothing is read).
__device__ __forceinline__ void cp_async_f32(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Launch accounting (profile.cu).  Construct a LaunchScope right before a
// kernel launch and let it go out of scope right after: it counts the launch,
// adds its algorithmic flops and bytes, and (when timing is enabled through
// ct_profile_enable) brackets it with CUDA events on the launching stream.
// ---------------------------------------------------------------------------
enum KernelClass {
  K_ZERO = 0, K_SIDDON, K_PANEL, K_VTC, K_TW, K_UPDATE, K_TRSM_DIAG, K_COPY, K_RANK,
  K_NORMS, K_ADD, K_GEMM_TN, K_AXPY, K_TC_GEMM, K_SPMM, K_TILE_RT, K_CONV, K_GATE, K_TC_UPDATE,
  K_QT_OUTER, K_INNER, K_TINV, K_COUNT
};

// Graph capture: launches made between begin and end are recorded into
// `GraphCounts` instead of the counters; each replay adds them back.
struct GraphCounts {
  uint64_t launches[K_COUNT];
  double flops[K_COUNT];
};
void profile_begin_capture();
void profile_end_capture(GraphCounts* out);
void profile_note_replay(const GraphCounts& c);

class LaunchScope {
 public:
  LaunchScope(int cls, cudaStream_t s, double flops = 0.0, double bytes = 0.0);
  ~LaunchScope();
  LaunchScope(const LaunchScope&) = delete;
  LaunchScope& operator=(const LaunchScope&) = delete;

 private:
  int cls_;
  cudaStream_t s_;
  void* start_;
};

// ---------------------------------------------------------------------------
// Device properties cached per process (device 0 of the current context).
// ---------------------------------------------------------------------------
struct DeviceInfo {
  int device = -1;
  int sms = 0;
  int smem_optin = 0;
};
ct_status device_info(DeviceInfo* out);

// ---------------------------------------------------------------------------
// The factor.
// ---------------------------------------------------------------------------
}  // namespace ctqr

struct ct_factor {
  int64_t m = 0, n = 0, ld = 0;
  int nb = 0;
  ct_prec prec = CT_PREC_F64;
  ct_dtype store = CT_F64;      // element type of F (FP64 for plain, FP32 otherwise)
  void* F = nullptr;            // factored matrix (R above, V below the diagonal)
  bool owns_F = true;
  double* tau = nullptr;        // n reflector scalars
  double* T = nullptr;          // npanels blocks of nb x nb (column-major, upper)
  int* status = nullptr;        // device status word
  unsigned long long* barrier = nullptr;  // grid-barrier counter
  double* partials = nullptr;   // panel-kernel reduction scratch
  size_t partials_elems = 0;
  int panel_cap = 0;            // when > 0: at most this many CTAs per panel launch
  float* Gblk = nullptr;        // two-level factors: V^T V of every 128-column outer
                                // block (128 x 128, strict upper part; blocks whose
                                // update ran, i.e. all but the last)
  float* Tblk = nullptr;        // the same blocks' compact-WY T = S^{-1} (128 x 128,
                                // column-major, upper)
  int device = 0;
  bool F_host = false;          // F is the caller's host matrix (ct_qr_factor_host):
                                // every use streams it through HBM
  int64_t ooc_bw = 0;           // host factors: block-column width of the streaming
  bool ooc_overlap = true;      // host factors: copies on their own stream
};

namespace ctqr {

// Factors whose outer trailing updates run on the tensor cores (two-level
// factors with per-128-column V^T V and T blocks).
inline bool tc_prec(ct_prec p) { return p == CT_PREC_TF32 || p == CT_PREC_F16X3; }

int64_t npanels(const ct_factor* f);
// Release a factor and every buffer it owns (no synchronisation).
void free_factor(ct_factor* f);
// Allocate tau, the panel T blocks, the status word, the barrier counters,
// the panel partials and (CT_PREC_TF32) the per-outer-block G and T stores
// for a factor whose m, n, nb and prec are set (api.cu).
ct_status alloc_factor_aux(ct_factor* f, const DeviceInfo& di);
// Allocate an owned factored matrix (ld = m rounded up to 4 elements).
ct_status alloc_factor_matrix(ct_factor* f);

// ---- system matrix (siddon.cu) --------------------------------------------
ct_status launch_build_system(const ct_geometry* g, ct_dtype dtype, double lambda, void* A,
                              int64_t lda, int64_t m, int64_t n, cudaStream_t s);

// ---- panel factorization (qr_panel.cu) ------------------------------------
// Factor the panel F[j0:m, j0:j0+nbp] in FP64, write V/R back in the storage
// type, tau[j0:j0+nbp] and the nbp x nbp upper T factor (ldt = nb).
ct_status launch_panel(ct_factor* f, int64_t j0, int nbp, double* T, cudaStream_t s);
size_t panel_partials_elems(int sms, int nb);

// ---- block-reflector application (gemm_simt.cu) ---------------------------
// C <- (I - V T V^T)^T C = C - V T^T V^T C for the mr x nc matrix C (leading
// dimension ldc, type of C given by c_f64), V = unit lower trapezoid of the
// panel at Fp (leading dimension ldf, storage type given by v_f64), nbp
// reflectors, T upper nbp x nbp (leading dimension ldt).  Uses `work`
// (at least reflector_work_elems(...) doubles).
struct ReflectorArgs {
  const void* V; bool v_f64; int64_t ldv;
  const double* T; int ldt;
  int nbp;
  void* C; bool c_f64; int64_t ldc;
  int64_t mr, nc;
  bool fp32_math;  // accumulate in FP32 (mixed factor) instead of FP64
  int max_splits = 0;  // cap on the row splits of V^T C (0: no cap)
};
size_t reflector_work_elems(int sms, int nbp, int64_t nc);
ct_status apply_block_reflector(const ReflectorArgs& a, double* work, size_t work_elems,
                                int sms, cudaStream_t s);

// C <- (I - V T V^T)^T C for the 128-column outer block [J, J + 128) of a
// two-level factor, T given through its UT-transform form S = T^{-1} =
// diag(1/tau) + striu(G), G = V^T V (gemm_simt.cu); work as for
// apply_block_reflector.
// One inner panel's block reflector (columns [j0, j0+nbp), T at Tp) applied to
// the columns [j0+nbp, cend) of an FP32-stored factor in one cooperative
// launch; CT_ERR_UNSUPPORTED (nothing launched) when the shape does not fit.
ct_status inner_update_persist(ct_factor* f, int64_t j0, int nbp, int64_t cend, const double* Tp, double* work,
                               size_t work_elems, int sms, cudaStream_t s);
// Q^T C (FP32 C and arithmetic, 1 <= k <= 32) for the outer blocks [0, nblk)
// of a two-level factor in one cooperative launch; CT_ERR_UNSUPPORTED when
// the factor or the shape does not allow it (nothing launched).
ct_status apply_qt_outer_persist(const ct_factor* f, float* C, int64_t ldc, int64_t k, int nblk, double* work,
                                 size_t work_elems, int sms, cudaStream_t s);
ct_status apply_outer_reflector(const ct_factor* f, int64_t J, void* C, bool c_f64, int64_t ldc, int64_t k,
                                bool fp32_math, double* work, size_t work_elems, int sms, cudaStream_t s);

// FP64 two-level factorization (gemm_simt.cu): the trailing update of the
// columns right of the nbo (<= 128) reflectors at column J, with a contraction
// over all nbo of them; work holds fp64_outer_work_elems(...) doubles.
size_t fp64_outer_work_elems(int sms, int64_t n);
ct_status fp64_outer_update(ct_factor* f, int64_t J, int nbo, double* work, size_t work_elems, int sms,
                            cudaStream_t s);

// Q^T C for all panels of the factor, in factorization order (api.cu).
ct_status apply_qt_all(const ct_factor* f, void* C, bool c_f64, int64_t ldc, int64_t k, bool fp32_math,
                       double* work, size_t work_elems, int sms, cudaStream_t s, int max_splits = 0);

// ---- out-of-core use of a host-resident factor (ooc.cu) -------------------
ct_status ooc_apply_qt(const ct_factor* f, double* B, int64_t ldb, int64_t k, cudaStream_t s);
ct_status ooc_trsm(const ct_factor* f, double* B, int64_t ldb, int64_t k, cudaStream_t s);

// ---- triangular solve (trsm.cu) -------------------------------------------
ct_status launch_trsm(const ct_factor* f, void* B, bool b_f64, int64_t ldb, int64_t k,
                      cudaStream_t s);
ct_status launch_dense_update(const void* V, bool v_f64, int64_t ldv, int K, const void* W,
                              int64_t ldw, void* C, bool b_f64, int64_t ldc, int64_t mr, int64_t nc,
                              cudaStream_t s);
int panel_width_that_fits(int64_t mr, int want, const DeviceInfo& di, size_t mth, bool pow2);
// Tensor-core update of C = F[J:m, J+nbo:n] with the 128-column block
// reflector of F[J:m, J:J+nbo] (outer_update.cu); work holds
// outer_work_floats(...) floats.
size_t outer_work_floats(int sms, int64_t m, int64_t n, int width);
// Look-ahead: the update of the columns after the next outer block runs on
// s2 (on all but `reserve` SMs) while the next block's panels run on s.
struct Lookahead {
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_w = nullptr, ev_rest = nullptr;
  // side stream for T = S^{-1}, which needs only V^T V and tau, so it runs
  // beside the V^T C product (ev_g: V^T V reduced; ev_t: T written)
  cudaStream_t s3 = nullptr;
  cudaEvent_t ev_g = nullptr, ev_t = nullptr;
  bool defer = false;         // defer the rest of this block's update
  bool rest_pending = false;  // a deferred update is in flight (ev_rest recorded)
  int reserve = 0;
};
ct_status outer_block_update(ct_factor* f, int64_t J, int nbo, float* work, size_t work_floats, int sms,
                             bool split3, cudaStream_t s, Lookahead* la = nullptr, int64_t cend = 0);
// The update of C = F[J:m, J+128+nbo_b:n] with the 256-column block reflector
// of F[J:m, J:J+128+nbo_b] (two 128-column halves, the first already applied
// to the second by outer_block_update(..., cend = J + 128 + nbo_b)); also
// forms the second half's V^T V and T blocks.  work: outer_work_floats(...,
// 256) floats.
ct_status outer_block_update256(ct_factor* f, int64_t J, int nbo_b, float* work, size_t work_floats, int sms,
                                bool split3, cudaStream_t s, Lookahead* la);
// ---- FP16-split outer updates (outer_update.cu, tc_f16.cu) ----------------
// Per-column bounds (float bits) on the trailing matrix's magnitudes: each
// column's 2-norm over the rows from the current outer block's first row
// down, which the orthogonal updates preserve, so it bounds every entry below
// any later block's first row.  The first block's come from one pass over the
// matrix; each later block's from the sums of squares that the previous
// block's V^T C product forms while it splits the trailing matrix (acc).
// bound and acc hold n entries each.
struct F16Cols {
  unsigned* bound = nullptr;
  double* acc = nullptr;
};
size_t outer_work_floats16(int sms, int64_t m, int64_t n, int width);
// cs->bound = the column norms of the FP32 factored matrix (the first block's).
ct_status f16_bounds(ct_factor* f, F16Cols* cs, cudaStream_t s);
// As outer_block_update / outer_block_update256 with the FP16-split products.
ct_status outer_update16(ct_factor* f, int64_t J, int nbo, float* work, size_t work_floats, int sms,
                         cudaStream_t s, Lookahead* la, int64_t cend, const F16Cols* cs);
ct_status outer_update256_16(ct_factor* f, int64_t J, int nbo_b, float* work, size_t work_floats, int sms,
                             cudaStream_t s, Lookahead* la, const F16Cols* cs);
// Whether a panel of mr rows and nbp columns fits on `ctas` CTAs (qr_panel.cu).
bool panel_fits_ctas(int64_t mr, int nbp, int ctas, const DeviceInfo& di);
ct_status launch_zero_matrix(void* A, size_t elem, int64_t lda, int64_t rows, int64_t cols,
                             cudaStream_t s);
ct_status launch_rank_check(ct_factor* f, cudaStream_t s);
// B[0:n] <- R^{-T} B[0:n] (FP64 B, or FP32 B with an FP32-stored R).
ct_status launch_trsm_t(const ct_factor* f, void* B, bool b_f64, int64_t ldb, int64_t k, cudaStream_t s);
// C(r, c) -= sum_{a<K} V(a, r) W(a, c) (V read transposed); W and C FP64 or FP32.
ct_status launch_dense_update_t(const void* V, bool v_f64, int64_t ldv, int K, const void* W, int64_t ldw,
                                void* C, bool b_f64, int64_t ldc, int64_t mr, int64_t nc, cudaStream_t s);
// Column-wise dot products out[c] = sum_r X[r, c] Y[r, c] (FP64).
ct_status launch_col_dots(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t rows,
                          int64_t k, double* out, cudaStream_t s);
// Y = A^T R: A m x n (FP64 or FP32), R m x k FP64, Y n x k FP64.
ct_status launch_gemm_tn(const void* A, bool a_f64, int64_t lda, const double* R, int64_t ldr,
                         double* Y, int64_t ldy, int64_t m, int64_t n, int64_t k, cudaStream_t s);
// Column-wise updates with per-column device scalars a[c] (a == NULL: 1):
//   mode 0: Y[:, c] += sign * a[c] * X[:, c];   mode 1: Y[:, c] = X[:, c] + a[c] * Y[:, c].
ct_status launch_colwise(int mode, double sign, const double* a, const double* X, int64_t ldx,
                         double* Y, int64_t ldy, int64_t rows, int64_t k, cudaStream_t s);

// ---- tensor-core GEMM (tc_gemm.cu) ---------------------------------------
// C (M x N) = A^T B (mode 0; split z of `splits` writes C + z*split_stride) or
// C -= A^T B (mode 1, splits must be 1); A is K x M, B is K x N, all FP32
// column-major, lda/ldb multiples of 4, A/B 16-byte aligned.  split3 selects
// error-compensated TF32 (hi*hi + hi*lo + lo*hi).
ct_status tc_gemm_tn(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M, int64_t N,
                     int64_t K, float* C, int64_t ldc, int64_t split_stride, int mode, int splits,
                     bool split3, int* status, cudaStream_t s);

// ---- sparse system matrix (sparse.cu) -------------------------------------
// CSR + CSC of the rays-only A of a geometry (same entries as the dense build),
// with staging buffers for products with up to kmax right-hand sides.
struct SparseSystem {
  int64_t m = 0, n = 0, nnz = 0, kmax = 0;
  int64_t* row_ptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  int64_t* col_ptr = nullptr;
  int* crow = nullptr;
  double* cval = nullptr;
  double* stage = nullptr;
  ~SparseSystem();
  void release();
  ct_status build(const ct_geometry* g, int64_t k_max, int* status, cudaStream_t s);
  // Y op= A X (mode 0 store, 1 subtract, 2 store negated); X n x k, Y m x k.
  ct_status apply(const double* X, int64_t ldx, int64_t k, double* Y, int64_t ldy, int mode,
                  cudaStream_t s) const;
  // S = A^T R; R m x k, S n x k.
  ct_status apply_t(const double* R, int64_t ldr, int64_t k, double* S, int64_t lds, cudaStream_t s) const;
};

// C (M x N) -= A^T B, persistent tensor-core kernel on operands split into
// TF32 high (Ah, Bh) and low (Al, Bl) parts (low parts unused unless split3).
ct_status tc_update_presplit(const float* Ah, const float* Al, int64_t lda, const float* Bh, const float* Bl,
                             int64_t ldb, int64_t M, int64_t N, int64_t K, float* C, int64_t ldc, bool split3,
                             int sms, int* status, cudaStream_t s);

// ---- batched tile QR (tile_qr.cu) and its autotuner (autotune.cu) --------
// Factor and solve `count` systems with the tile-task runtime, tile b = 32 or
// 64; *ms_out receives the device time of the persistent launch.  keep: the
// task list, T blocks and instantiated graph stay on the device for the next
// call with the same sizes (one shape per process; release_batch_cache frees
// it); otherwise everything is released before returning.
ct_status run_batch(int count, const ct_batch_system* in, int tile, int sms, int* status, cudaStream_t s,
                    bool keep, double* ms_out, int* tasks_out = nullptr);
void release_batch_cache();
// The task list plan_batch builds (host only): kPlanRecord int32 per task,
// see ct_batch_plan in ctqr.h.
constexpr int kPlanRecord = 25;
ct_status export_batch_plan(int count, const ct_batch_system* in, int tile, int32_t* out, int64_t max_tasks,
                            int64_t* ntasks, int* nparts);
// Tile tasks the batch would hold with tile size b (each task is ~100 bytes
// of host and device memory).
int64_t batch_task_count(int count, const ct_batch_system* in, int b);
// Panel width and outer-block width of a tensor-core factorization of an
// m x n matrix (CT_PREC_TF32 with `passes` TF32 passes, or CT_PREC_F16X3,
// whose outer width stays 256): cached choice, or measured now on a synthetic
// matrix (CTQR_NO_TUNE=1: the defaults 32 and 256).
ct_status tuned_factor_widths(int64_t m, int64_t n, int passes, ct_prec prec, cudaStream_t s, int* nb, int* outer);
// Tile size for systems of this shape: cached choice, or measured now.
ct_status tuned_batch_tile(int64_t m, int64_t n, int sms, cudaStream_t s, int* tile);

// ---- surrogate convolutions on the tensor cores (conv_tc.cu) -------------
}  // namespace ctqr
#include <cuda_bf16.h>
#include <cuda_fp16.h>
namespace ctqr {
// ---- FP16-split tensor-core products (tc_f16.cu) ---------------------------
// W (M x N) = A^T B with A (K x M) given as FP16 parts Ah + Al (ld lda, a
// multiple of 8) and B either FP32 (Bl == NULL; ldb a multiple of 4; split
// on chip with per-column scales from bmax, bounds on its columns'
// magnitudes as float bits) or FP16 parts (Bh, Bl; ldb a multiple of 8); every output
// multiplied by out_scale (and by the inverse column scale for FP32 B).
// Split z of `splits` over K writes C + z * split_stride; *made = splits made.
ct_status tc_gemm16(const __half* Ah, const __half* Al, int64_t lda, const void* Bh, const __half* Bl, int64_t ldb,
                    const unsigned* bmax, double* nrm2, int64_t M, int64_t N, int64_t K, float out_scale, float* C,
                    int64_t ldc, int64_t split_stride, int splits, int* status, cudaStream_t s, int* made);
// CTAs tc_gemm16 puts on the M rows of one column tile for FP32 B.
int tc_gemm16_m_ctas(int64_t M);
// C (M x N) -= colinv[c] * (A^T B)[:, c] on FP16 parts (ld multiples of 8,
// K <= 256; colinv 16-byte aligned and readable up to N rounded up to 128).
ct_status tc_update16(const __half* Ah, const __half* Al, int64_t lda, const __half* Bh, const __half* Bl, int64_t ldb,
                      const float* colinv, int64_t M, int64_t N, int64_t K, float* C, int64_t ldc, int sms, int* status,
                      cudaStream_t s);
// bound[c] = bits of a float above sqrt(nrm2[c]).
ct_status launch_norm_bound(const double* nrm2, int64_t cols, unsigned* bound, cudaStream_t s);
// bound[c] = bits of a float above ||X[0:rows, c]||_2 (acc: cols doubles of scratch).
ct_status launch_colnorm_bound(const float* X, int64_t ldx, int64_t rows, int64_t cols, double* acc, unsigned* bound,
                               cudaStream_t s);
// FP16 parts H + L = s X (K x cols, ld ldo) with s = 2^exp_fixed, or per column
// from cmax (a bound on its magnitudes, below 2^14 after scaling);
// colinv[c] = 1 / (s_c 2^extra_exp).
ct_status launch_split16(const float* X, int64_t ldx, int64_t K, int64_t cols, const unsigned* cmax, int exp_fixed,
                         int extra_exp, __half* H, __half* L, int64_t ldo, float* colinv, cudaStream_t s);
ct_status launch_conv_tc(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias, int H, int W, int64_t B,
                         const __nv_bfloat16* res, __nv_bfloat16* r_out, __nv_bfloat16* a_out, int* status,
                         cudaStream_t s);

// ---- solve through a factor (api.cu) ---------------------------------------
// X = solution of the system f factors for the right-hand sides B (f->m rows):
// the plain FP64 apply + back-solve when sp is NULL, else FP64-residual
// refinement with the exact sparse A (rays only; ropts->lambda adds the
// implicit lambda*I rows).
ct_status reconstruct_with(const ct_factor* f, const SparseSystem* sp, const double* B, int64_t ldb, double* X,
                           int64_t ldx, int64_t k, const ct_refine_opts* ropts, ct_report* report, cudaStream_t s);

// ---- utilities (util.cu) ---------------------------------------------------
ct_status launch_copy_matrix(const void* src, ct_dtype st, int64_t lds, void* dst, ct_dtype dt,
                             int64_t ldd, int64_t rows, int64_t cols, cudaStream_t s);
// Per-column reductions and updates used by the refinement (refine.cu).
ct_status launch_col_norms2(const double* X, int64_t ldx, int64_t rows, int64_t k, double* out,
                            cudaStream_t s);
// X[0:rows, 0:k] += D; dnorm2[c] = ||D_c||^2, xnorm2[c] = ||X_c||^2 afterwards.
ct_status launch_add_f32_to_f64(const float* D, int64_t ldd, double* X, int64_t ldx, int64_t rows,
                                int64_t k, double* dnorm2, double* xnorm2, cudaStream_t s);
ct_status launch_add_f64_to_f64(const double* D, int64_t ldd, double* X, int64_t ldx, int64_t rows,
                                int64_t k, double* dnorm2, double* xnorm2, cudaStream_t s);

}  // namespace ctqr
