// api.cu -- the C ABI of include/ctqr.h: argument checks, the factor's
// lifetime, and the host-side sequencing of the kernels on the caller's stream.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "internal.cuh"

using namespace ctqr;

namespace {

inline cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

bool geometry_ok(const ct_geometry* g) {
  if (!g) return false;
  if (g->beam != 0 && g->beam != 1) return false;
  if (g->nx < 1 || g->ny < 1 || g->n_views < 1 || g->n_bins < 1) return false;
  if (!(g->pixel > 0.0) || !isfinite(g->pixel)) return false;
  if (!isfinite(g->angle0) || !isfinite(g->angle_span) || !isfinite(g->det_span)) return false;
  if (g->beam == 1 && !(g->src_iso > 0.0 && isfinite(g->src_iso))) return false;
  if (g->angle_rule != 0 && g->angle_rule != 1) return false;
  const double half = 0.5 * sqrt((double)g->nx * g->nx + (double)g->ny * g->ny) * g->pixel;
  if (g->beam == 1 && g->src_iso <= half) return false;  // source inside the image
  return true;
}

// Stream-ordered scratch that frees itself.
struct Scratch {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  ct_status alloc(size_t bytes, cudaStream_t st) {
    s = st;
    if (bytes == 0) bytes = 16;
    if (getenv("CTQR_FAULT_NOMEM")) return CT_ERR_NOMEM;  // host-side fault injection
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? CT_ERR_NOMEM : CT_ERR_CUDA;
    }
    return CT_OK;
  }
  ~Scratch() {
    if (p) cudaFreeAsync(p, s);
  }
};

template <typename T>
ct_status dev_alloc(T** p, size_t elems) {
  if (getenv("CTQR_FAULT_NOMEM")) return CT_ERR_NOMEM;
  cudaError_t e = cudaMalloc((void**)p, elems * sizeof(T) + 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? CT_ERR_NOMEM : CT_ERR_CUDA;
  }
  return CT_OK;
}

size_t elem_size(ct_dtype t) { return t == CT_F64 ? 8 : 4; }

ct_status read_status(const ct_factor* f, cudaStream_t s) {
  int h = 0;
  CT_CUDA_TRY(cudaMemcpyAsync(&h, f->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CT_CUDA_TRY(cudaStreamSynchronize(s));
  return (ct_status)h;
}


// FP64-residual refinement of X for a factor of A (see ct_reconstruct_batch).
// A is the dense matrix the caller passed, or the sparse form of the system
// built from a geometry (ct_reconstruct_scan); either way every product with
// A or A^T is exact FP64.
class Refiner {
 public:
  Refiner(const ct_factor* f, const void* A, ct_dtype adt, int64_t lda, const SparseSystem* sp, const double* B,
          int64_t ldb, double* X, int64_t ldx, int64_t k, cudaStream_t s, int sms)
      : f_(f), A_(A), a64_(adt == CT_F64), lda_(lda), sp_(sp), B_(B), ldb_(ldb), X_(X), ldx_(ldx), k_(k),
        s_(s), sms_(sms), m_(f->m), n_(f->n), ldw_((f->m + 3) / 4 * 4) {}

  ct_status run(const ct_refine_opts* o, ct_report* rep) {
    // Work on a private stream ordered after the caller's (graph capture is
    // not allowed on the legacy default stream); the caller's stream waits
    // for it at the end.
    ct_status st0 = own_.attach(s_);
    if (st0 != CT_OK) return st0;
    s_ = own_.s;
    ct_status r = run_inner(o, rep);
    own_.detach();
    return r;
  }

  ct_status run_inner(const ct_refine_opts* o, ct_report* rep) {
    const int max_iter = o && o->max_iter > 0 ? o->max_iter : 200;
    tol_ = o && o->tol > 0.0 ? o->tol : 1e-12;
    lam_ = o && o->lambda > 0.0 ? o->lambda : 0.0;
    ma_ = lam_ > 0.0 ? m_ - n_ : m_;
    if (ma_ < 0) return CT_ERR_INVALID;
    if (sp_ && (sp_->m != ma_ || sp_->n != n_)) return CT_ERR_INVALID;
    const int method = o ? o->method : 0;
    ct_status st;
    if ((st = alloc()) != CT_OK) return st;
    if ((st = launch_col_norms2(B_, ldb_, m_, k_, bn2_, s_)) != CT_OK) return st;
    // X_0 = R^{-1} (Q^T B)[0:n], then classical corrections while they pay.
    if ((st = launch_zero_matrix(X_, 8, ldx_, n_, k_, s_)) != CT_OK) return st;
    int it = 0;
    double prev = INFINITY;
    ct_status result = CT_ERR_NOCONVERGE;
    // lambda*I rows make the system inconsistent: go to CGLS after X_0.
    const bool classical_only = method == 1;
    const bool cgls_now = method == 2 || (method == 0 && lam_ > 0.0);
    bool go_cgls = false, have_residual = false;
    for (; it <= max_iter; ++it) {
      double worst = 0.0;
      // The residual of X_0 tells whether B is consistent: a residual well
      // above rounding level means noisy data, where only CGLS reaches the
      // least-squares solution, so it goes there without a classical step.
      int mode = it == 0 ? 0 : 1;
      if (it == 1 && method == 0) {
        if ((st = residual_norm()) != CT_OK) return st;
        if (resid_ > 1e-6) {
          if (trace_) fprintf(stderr, "ctqr residual of X_0 %.3e: to CGLS (%.2f ms)\n", resid_, since_start());
          go_cgls = true;
          have_residual = true;
          break;
        }
        mode = 2;
      }
      if ((st = classical_step(mode, &worst)) != CT_OK) return st;
      if (it == 0) {
        if (trace_) fprintf(stderr, "ctqr X_0 = R^-1 (Q^T B) (%.2f ms)\n", since_start());
        if (cgls_now) { go_cgls = true; break; }
        continue;
      }
      last_ = worst;
      if (trace_) fprintf(stderr, "ctqr classical %d: max |dx|/|x| = %.3e (%.2f ms)\n", it, worst, since_start());
      if (worst <= tol_) { result = CT_OK; break; }
      if (!isfinite(worst)) return CT_ERR_NONFINITE;
      if (!classical_only && it >= 2 && worst > 0.25 * prev) { go_cgls = true; break; }
      prev = worst;
    }
    if (go_cgls) {
      int used = 0;
      result = cgls(max_iter - it, &used, have_residual);
      it += used;
    }
    if (rep) {
      rep->iterations = it > max_iter ? max_iter : it;
      rep->last_update = last_;
      rep->residual = resid_;
    }
    return result;
  }

 private:
  // A non-blocking stream that follows `parent` (declared first: destroyed
  // after the scratch buffers whose frees are queued on it).
  struct OwnStream {
    cudaStream_t s = nullptr, parent = nullptr;
    cudaEvent_t ev = nullptr;
    ct_status attach(cudaStream_t p) {
      parent = p;
      CT_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      CT_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      CT_CUDA_TRY(cudaEventRecord(ev, parent));
      CT_CUDA_TRY(cudaStreamWaitEvent(s, ev, 0));
      return CT_OK;
    }
    void detach() {
      if (s && ev && cudaEventRecord(ev, s) == cudaSuccess) cudaStreamWaitEvent(parent, ev, 0);
    }
    ~OwnStream() {
      if (ev) cudaEventDestroy(ev);
      if (s) cudaStreamDestroy(s);
    }
  } own_;
  const ct_factor* f_;
  const void* A_;
  bool a64_;
  int64_t lda_;
  const SparseSystem* sp_;
  const double* B_;
  int64_t ldb_;
  double* X_;
  int64_t ldx_, k_;
  cudaStream_t s_;
  int sms_;
  int64_t m_, n_, ldw_;
  double tol_ = 1e-12, last_ = INFINITY, resid_ = 0.0, lam_ = 0.0;
  int64_t ma_ = 0;  // rows of A (the lambda*I rows below it are implicit)
  size_t work_elems_ = 0;
  Scratch work_, Y_, D_, cg_, scal_;
  double *Yd_ = nullptr, *bn2_ = nullptr, *n1_ = nullptr, *n2_ = nullptr, *n3_ = nullptr, *a_ = nullptr;
  double *S_ = nullptr, *P_ = nullptr, *T_ = nullptr, *Q_ = nullptr, *S0_ = nullptr;
  std::vector<double> h_;

  bool f32() const { return f_->store == CT_F32; }
  // Diagnostics: CTQR_TRACE=1 prints every step's update size to stderr;
  // CTQR_PRECOND_F64=1 runs the preconditioner solves in FP64 arithmetic.
  bool trace_ = getenv("CTQR_TRACE") != nullptr;
  std::chrono::steady_clock::time_point t0_ = std::chrono::steady_clock::now();
  // host milliseconds since the refinement started (trace output only)
  double since_start() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0_).count();
  }
  bool precond_f64_ = getenv("CTQR_PRECOND_F64") != nullptr;

  ct_status alloc() {
    ct_status st;
    work_elems_ = reflector_work_elems(sms_, f_->nb, k_);
    if ((st = work_.alloc(work_elems_ * sizeof(double), s_)) != CT_OK) return st;
    if ((st = Y_.alloc((size_t)ldw_ * k_ * sizeof(double), s_)) != CT_OK) return st;
    if (f32() && (st = D_.alloc((size_t)ldw_ * k_ * sizeof(float), s_)) != CT_OK) return st;
    if ((st = scal_.alloc((size_t)5 * k_ * sizeof(double), s_)) != CT_OK) return st;
    Yd_ = (double*)Y_.p;
    bn2_ = (double*)scal_.p;
    n1_ = bn2_ + k_;
    n2_ = n1_ + k_;
    n3_ = n2_ + k_;
    a_ = n3_ + k_;
    h_.resize((size_t)4 * k_);
    return CT_OK;
  }

  ct_status fetch(const double* d, int count) {
    CT_CUDA_TRY(cudaMemcpyAsync(h_.data(), d, sizeof(double) * k_ * count, cudaMemcpyDeviceToHost, s_));
    CT_CUDA_TRY(cudaStreamSynchronize(s_));
    return CT_OK;
  }

  // Yd[0:ma] -= A X.
  ct_status sub_AX(const double* X, int64_t ldx) {
    if (sp_) return sp_->apply(X, ldx, k_, Yd_, ldw_, 1, s_);
    return launch_dense_update(A_, a64_, lda_, (int)n_, X, ldx, Yd_, true, ldw_, ma_, k_, s_);
  }

  // Q = [A; lambda I] T.
  ct_status mul_A(const double* T, int64_t ldt, double* Q) {
    ct_status st;
    if (sp_) {
      if ((st = sp_->apply(T, ldt, k_, Q, ldw_, 0, s_)) != CT_OK) return st;
    } else {
      if ((st = launch_zero_matrix(Q, 8, ldw_, ma_, k_, s_)) != CT_OK) return st;
      if ((st = launch_dense_update(A_, a64_, lda_, (int)n_, T, ldt, Q, true, ldw_, ma_, k_, s_)) != CT_OK) return st;
      if ((st = scale_neg(Q, ma_)) != CT_OK) return st;  // the update left -A T in Q
    }
    if (lam_ > 0.0) {
      if ((st = launch_zero_matrix(Q + ma_, 8, ldw_, n_, k_, s_)) != CT_OK) return st;
      if ((st = launch_colwise(0, lam_, nullptr, T, ldt, Q + ma_, ldw_, n_, k_, s_)) != CT_OK) return st;
    }
    return CT_OK;
  }

  ct_status scale_neg(double* Q, int64_t rows) {
    // Q = -Q via Q += (-2) Q.
    return launch_colwise(0, -2.0, nullptr, Q, ldw_, Q, ldw_, rows, k_, s_);
  }

  // Res = B - [A; lambda I] X into Yd (m x k).
  ct_status residual() {
    ct_status st;
    if ((st = launch_copy_matrix(B_, CT_F64, ldb_, Yd_, CT_F64, ldw_, m_, k_, s_)) != CT_OK) return st;
    if ((st = sub_AX(X_, ldx_)) != CT_OK) return st;
    if (lam_ > 0.0) return launch_colwise(0, -lam_, nullptr, X_, ldx_, Yd_ + ma_, ldw_, n_, k_, s_);
    return CT_OK;
  }

  // Res = B - [A; lambda I] X into Yd, its column norms into n1 and
  // resid_ = ||Res||_F / ||B||_F.
  ct_status residual_norm() {
    ct_status st;
    if ((st = residual()) != CT_OK) return st;
    if ((st = launch_col_norms2(Yd_, ldw_, m_, k_, n1_, s_)) != CT_OK) return st;
    if ((st = fetch(bn2_, 2)) != CT_OK) return st;
    double rr = 0.0, bb = 0.0;
    for (int64_t c = 0; c < k_; ++c) {
      bb += h_[c];
      rr += h_[k_ + c];
    }
    resid_ = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
    return CT_OK;
  }

  // One classical step: mode 0 is the first solve (X = 0), mode 1 forms the
  // residual of X first, mode 2 takes the residual (and its norms) that
  // residual_norm() left in Yd.
  ct_status classical_step(int mode, double* worst) {
    ct_status st;
    const bool with_residual = mode != 0;
    if (mode == 1) {
      if ((st = residual()) != CT_OK) return st;
      if ((st = launch_col_norms2(Yd_, ldw_, m_, k_, n1_, s_)) != CT_OK) return st;
    } else if (mode == 0) {
      if ((st = launch_copy_matrix(B_, CT_F64, ldb_, Yd_, CT_F64, ldw_, m_, k_, s_)) != CT_OK) return st;
    }
    if (f32()) {
      float* D = (float*)D_.p;
      if ((st = launch_copy_matrix(Yd_, CT_F64, ldw_, D, CT_F32, ldw_, m_, k_, s_)) != CT_OK) return st;
      if ((st = apply_qt_all(f_, D, false, ldw_, k_, true, (double*)work_.p, work_elems_, sms_, s_)) != CT_OK) return st;
      if ((st = launch_trsm(f_, D, false, ldw_, k_, s_)) != CT_OK) return st;
      if ((st = launch_add_f32_to_f64(D, ldw_, X_, ldx_, n_, k_, n2_, n3_, s_)) != CT_OK) return st;
    } else {
      if ((st = apply_qt_all(f_, Yd_, true, ldw_, k_, false, (double*)work_.p, work_elems_, sms_, s_)) != CT_OK) return st;
      if ((st = launch_trsm(f_, Yd_, true, ldw_, k_, s_)) != CT_OK) return st;
      if ((st = launch_add_f64_to_f64(Yd_, ldw_, X_, ldx_, n_, k_, n2_, n3_, s_)) != CT_OK) return st;
    }
    // h = [bn2 | n1 = ||res||^2 | n2 = ||d||^2 | n3 = ||x||^2]
    if ((st = fetch(bn2_, 4)) != CT_OK) return st;
    double w = 0.0, rr = 0.0, bb = 0.0;
    for (int64_t c = 0; c < k_; ++c) {
      const double xc = sqrt(h_[3 * k_ + c]), dc = sqrt(h_[2 * k_ + c]);
      const double rel = xc > 0.0 ? dc / xc : (dc > 0.0 ? INFINITY : 0.0);
      if (!(rel <= w)) w = rel;
      rr += h_[k_ + c];
      bb += h_[c];
    }
    if (with_residual) resid_ = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
    *worst = w;
    return CT_OK;
  }

  // A captured sequence of launches replayed as one CUDA graph.
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    bool failed = false;
    GraphCounts counts{};
    ~Graph() {
      if (exec) cudaGraphExecDestroy(exec);
    }
  };
  Graph g_solve_, g_solve_t_;

  // The preconditioner solve on the fixed buffer Z, captured into a graph on
  // first use (hundreds of small launches) and replayed afterwards.
  ct_status precond_graph(double* Z, bool transpose, Graph& g) {
    if (getenv("CTQR_NO_GRAPHS")) return precond(Z, transpose);
    if (!g.exec && !g.failed) {
      cudaGraph_t graph = nullptr;
      profile_begin_capture();
      cudaError_t e = cudaStreamBeginCapture(s_, cudaStreamCaptureModeRelaxed);
      ct_status st = e == cudaSuccess ? precond(Z, transpose) : CT_ERR_CUDA;
      cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(s_, &graph) : e;
      profile_end_capture(&g.counts);
      if (st != CT_OK || e2 != cudaSuccess || !graph ||
          cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        g.exec = nullptr;
        g.failed = true;
      }
      if (graph) cudaGraphDestroy(graph);
      if (trace_) fprintf(stderr, "ctqr: preconditioner solve %s graph %s\n", transpose ? "R^-T" : "R^-1",
                          g.exec ? "captured" : "capture failed, launching directly");
      if (!g.exec) return precond(Z, transpose);
    }
    if (!g.exec) return precond(Z, transpose);
    LaunchScope ls(K_TRSM_DIAG, s_, 0.0, 0.0);
    CT_CUDA_TRY(cudaGraphLaunch(g.exec, s_));
    profile_note_replay(g.counts);
    return CT_OK;
  }

  // In-place preconditioner solves on an n x k FP64 block (ld n): R^{-1}
  // (transpose = false) or R^{-T}; FP32 arithmetic for an FP32-stored R.
  ct_status precond(double* Z, bool transpose) {
    ct_status st;
    if (!f32() || precond_f64_)
      return transpose ? launch_trsm_t(f_, Z, true, n_, k_, s_) : launch_trsm(f_, Z, true, n_, k_, s_);
    float* D = (float*)D_.p;
    if ((st = launch_copy_matrix(Z, CT_F64, n_, D, CT_F32, n_, n_, k_, s_)) != CT_OK) return st;
    if ((st = transpose ? launch_trsm_t(f_, D, false, n_, k_, s_) : launch_trsm(f_, D, false, n_, k_, s_)) != CT_OK)
      return st;
    return launch_copy_matrix(D, CT_F32, n_, Z, CT_F64, n_, n_, k_, s_);
  }

  // S = R^{-T} ([A; lambda I]^T r)  with r in Yd.
  ct_status precond_grad(double* S) {
    ct_status st;
    if (sp_) {
      if ((st = sp_->apply_t(Yd_, ldw_, k_, S, n_, s_)) != CT_OK) return st;
    } else if ((st = launch_gemm_tn(A_, a64_, lda_, Yd_, ldw_, S, n_, ma_, n_, k_, s_)) != CT_OK) {
      return st;
    }
    if (lam_ > 0.0 && (st = launch_colwise(0, lam_, nullptr, Yd_ + ma_, ldw_, S, n_, n_, k_, s_)) != CT_OK) return st;
    return precond_graph(S, true, g_solve_t_);
  }

  // Flexible preconditioned CGLS on min ||[A; lambda I] x - B|| from the
  // current X, the low-precision R as right preconditioner.  x and the
  // residual r are kept consistent in FP64 (r -= alpha A t with the exact
  // product of the very t added to x); alpha is the exact line search
  // <r, A t> / ||A t||^2 and beta the Polak-Ribiere ratio, so rounding in the
  // preconditioner solves slows the iteration but cannot move its fixed
  // point, A^T r = 0.
  ct_status cgls(int budget, int* used, bool have_residual) {
    ct_status st;
    *used = 0;
    if ((st = cg_.alloc(((size_t)5 * n_ * k_ + (size_t)ldw_ * k_) * sizeof(double), s_)) != CT_OK) return st;
    S_ = (double*)cg_.p;
    S0_ = S_ + n_ * k_;
    P_ = S0_ + n_ * k_;
    T_ = P_ + n_ * k_;
    double* G = T_ + n_ * k_;  // scratch n x k
    Q_ = G + n_ * k_;
    (void)G;
    if (!have_residual && (st = residual()) != CT_OK) return st;  // r = B - A X
    if ((st = precond_grad(S_)) != CT_OK) return st;        // s = R^-T A^T r
    if ((st = launch_copy_matrix(S_, CT_F64, n_, P_, CT_F64, n_, n_, k_, s_)) != CT_OK) return st;
    if ((st = launch_col_norms2(S_, n_, n_, k_, n1_, s_)) != CT_OK) return st;
    if ((st = fetch(n1_, 1)) != CT_OK) return st;
    std::vector<double> gamma(h_.begin(), h_.begin() + k_), alpha(k_), beta(k_);
    std::vector<double> prel(k_, 0.0), pratio(k_, INFINITY);  // last step and contraction per column
    for (int it = 0; it < budget; ++it) {
      *used = it + 1;
      // t = R^{-1} p ; q = [A; lambda I] t
      if ((st = launch_copy_matrix(P_, CT_F64, n_, T_, CT_F64, n_, n_, k_, s_)) != CT_OK) return st;
      if ((st = precond_graph(T_, false, g_solve_)) != CT_OK) return st;
      if ((st = mul_A(T_, n_, Q_)) != CT_OK) return st;
      if ((st = launch_col_dots(Yd_, ldw_, Q_, ldw_, m_, k_, n1_, s_)) != CT_OK) return st;   // <r, q>
      if ((st = launch_col_norms2(Q_, ldw_, m_, k_, n2_, s_)) != CT_OK) return st;           // ||q||^2
      if ((st = launch_col_norms2(T_, n_, n_, k_, n3_, s_)) != CT_OK) return st;             // ||t||^2
      if ((st = launch_col_norms2(X_, ldx_, n_, k_, a_, s_)) != CT_OK) return st;            // ||x||^2
      if ((st = fetch(n1_, 4)) != CT_OK) return st;
      // worst: max over columns of |dx|/|x|; est: max over columns of the
      // error left after this step, |dx| rho / (1 - rho) with rho the larger
      // of the last two contraction ratios |dx_t| / |dx_{t-1}| (the remaining
      // steps of an iteration contracting by rho sum to that), once two
      // ratios exist and both are below 1/2; otherwise the step itself.
      double worst = 0.0, est = 0.0;
      for (int64_t c = 0; c < k_; ++c) {
        const double rq = h_[c], qq = h_[k_ + c], tt = h_[2 * k_ + c], xx = h_[3 * k_ + c];
        alpha[c] = qq > 0.0 ? rq / qq : 0.0;
        const double dx = fabs(alpha[c]) * sqrt(tt), xn = sqrt(xx + alpha[c] * alpha[c] * tt);
        const double rel = xn > 0.0 ? dx / xn : (dx > 0.0 ? INFINITY : 0.0);
        if (!(rel <= worst)) worst = rel;
        double e = rel;
        const double ratio = prel[c] > 0.0 ? rel / prel[c] : INFINITY;
        if (it >= 2) {
          const double rho = ratio > pratio[c] ? ratio : pratio[c];
          if (rho < 0.5) e = rel * rho / (1.0 - rho);
        }
        pratio[c] = ratio;
        prel[c] = rel;
        if (!(e <= est)) est = e;
      }
      CT_CUDA_TRY(cudaMemcpyAsync(a_, alpha.data(), sizeof(double) * k_, cudaMemcpyHostToDevice, s_));
      if ((st = launch_colwise(0, 1.0, a_, T_, n_, X_, ldx_, n_, k_, s_)) != CT_OK) return st;    // x += a t
      if ((st = launch_colwise(0, -1.0, a_, Q_, ldw_, Yd_, ldw_, m_, k_, s_)) != CT_OK) return st;  // r -= a q
      last_ = worst;
      if (trace_)
        fprintf(stderr, "ctqr cgls %d: max |dx|/|x| = %.3e, estimated error left %.3e (%.2f ms)\n", it, worst, est,
                since_start());
      if (!isfinite(worst)) return CT_ERR_NONFINITE;
      if (worst <= tol_ || est <= tol_) {
        CT_CUDA_TRY(cudaStreamSynchronize(s_));
        return CT_OK;
      }
      // s_new = R^-T A^T r ; beta = <s_new, s_new - s_old> / gamma (Polak-Ribiere, >= 0)
      if ((st = launch_copy_matrix(S_, CT_F64, n_, S0_, CT_F64, n_, n_, k_, s_)) != CT_OK) return st;
      if ((st = precond_grad(S_)) != CT_OK) return st;
      if ((st = launch_col_norms2(S_, n_, n_, k_, n1_, s_)) != CT_OK) return st;
      if ((st = launch_col_dots(S_, n_, S0_, n_, n_, k_, n2_, s_)) != CT_OK) return st;
      if ((st = fetch(n1_, 2)) != CT_OK) return st;
      for (int64_t c = 0; c < k_; ++c) {
        const double ss = h_[c], s0 = h_[k_ + c];
        double b = gamma[c] > 0.0 ? (ss - s0) / gamma[c] : 0.0;
        beta[c] = b > 0.0 ? b : 0.0;
        gamma[c] = ss;
      }
      CT_CUDA_TRY(cudaMemcpyAsync(a_, beta.data(), sizeof(double) * k_, cudaMemcpyHostToDevice, s_));
      if ((st = launch_colwise(1, 1.0, a_, S_, n_, P_, n_, n_, k_, s_)) != CT_OK) return st;     // p = s + b p
    }
    return CT_ERR_NOCONVERGE;
  }
};

}  // namespace

namespace ctqr {
int64_t npanels(const ct_factor* f) { return (f->n + f->nb - 1) / f->nb; }

void free_factor(ct_factor* f) {
  if (!f) return;
  if (f->owns_F && f->F) cudaFree(f->F);
  if (f->tau) cudaFree(f->tau);
  if (f->T) cudaFree(f->T);
  if (f->status) cudaFree(f->status);
  if (f->barrier) cudaFree(f->barrier);
  if (f->partials) cudaFree(f->partials);
  if (f->Gblk) cudaFree(f->Gblk);
  if (f->Tblk) cudaFree(f->Tblk);
  delete f;
}

ct_status alloc_factor_aux(ct_factor* f, const DeviceInfo& di) {
  const bool tc = tc_prec(f->prec);
  const int64_t n = f->n, np = npanels(f);
  f->partials_elems = panel_partials_elems(di.sms, f->nb);
  ct_status st;
  if ((st = dev_alloc(&f->tau, (size_t)n)) != CT_OK ||
      (st = dev_alloc(&f->T, (size_t)np * f->nb * f->nb)) != CT_OK ||
      (st = dev_alloc(&f->status, 1)) != CT_OK ||
      (st = dev_alloc(&f->barrier, 3)) != CT_OK ||
      (st = dev_alloc(&f->partials, f->partials_elems)) != CT_OK ||
      (tc && (st = dev_alloc(&f->Gblk, (size_t)((n + 127) / 128) * 128 * 128)) != CT_OK) ||
      (tc && (st = dev_alloc(&f->Tblk, (size_t)((n + 127) / 128) * 128 * 128)) != CT_OK))
    return st;
  return CT_OK;
}

ct_status alloc_factor_matrix(ct_factor* f) {
  f->owns_F = true;
  f->ld = (f->m + 3) / 4 * 4;
  return dev_alloc((char**)&f->F, (size_t)f->ld * f->n * (f->store == CT_F64 ? 8 : 4));
}

// Apply Q^T (all panels, factorization order) to the mr = m rows of C (k
// columns, element type c_f64 ? FP64 : FP32).
ct_status apply_qt_all(const ct_factor* f, void* C, bool c_f64, int64_t ldc, int64_t k, bool fp32_math,
                       double* work, size_t work_elems, int sms, cudaStream_t s, int max_splits) {
  if (f->F_host) {  // a host-resident factor streams through HBM
    if (!c_f64 || fp32_math || max_splits) return CT_ERR_UNSUPPORTED;
    return ooc_apply_qt(f, (double*)C, ldc, k, s);
  }
  const size_t es = elem_size(f->store), cs = c_f64 ? 8 : 4;
  // Two-level factors apply each 128-column outer block at once (its panels'
  // reflectors in the same order), except the last block, whose V^T V the
  // factorization did not form; the allocation-free path (max_splits) keeps
  // the per-panel application.
  int64_t jblk = 0;
  if (f->Gblk && max_splits == 0) {
    // FP32 right-hand sides: all outer blocks in one persistent launch when it fits
    if (!c_f64 && fp32_math) {
      int nblk = 0;
      while ((int64_t)(nblk + 1) * 128 < f->n) ++nblk;
      ct_status st = nblk > 0 ? apply_qt_outer_persist(f, (float*)C, ldc, k, nblk, work, work_elems, sms, s)
                              : CT_ERR_UNSUPPORTED;
      if (st == CT_OK) jblk = (int64_t)nblk * 128;
      else if (st != CT_ERR_UNSUPPORTED) return st;
    }
    for (; jblk + 128 < f->n; jblk += 128) {
      ct_status st = apply_outer_reflector(f, jblk, (char*)C + (size_t)jblk * cs, c_f64, ldc, k, fp32_math, work,
                                           work_elems, sms, s);
      if (st != CT_OK) return st;
    }
  }
  for (int64_t j0 = jblk, p = jblk / f->nb; j0 < f->n; j0 += f->nb, ++p) {
    const int nbp = (int)(f->n - j0 < f->nb ? f->n - j0 : f->nb);
    ReflectorArgs a;
    a.V = (const char*)f->F + (size_t)(j0 + j0 * f->ld) * es;
    a.v_f64 = f->store == CT_F64;
    a.ldv = f->ld;
    a.T = f->T + (size_t)p * f->nb * f->nb;
    a.ldt = f->nb;
    a.nbp = nbp;
    a.C = (char*)C + (size_t)j0 * cs;
    a.c_f64 = c_f64;
    a.ldc = ldc;
    a.mr = f->m - j0;
    a.nc = k;
    a.fp32_math = fp32_math;
    a.max_splits = max_splits;
    ct_status st = apply_block_reflector(a, work, work_elems, sms, s);
    if (st != CT_OK) return st;
  }
  return CT_OK;
}

}  // namespace ctqr

extern "C" {

const char* ct_status_str(ct_status s) {
  switch (s) {
    case CT_OK: return "CT_OK";
    case CT_ERR_INVALID: return "CT_ERR_INVALID";
    case CT_ERR_NOMEM: return "CT_ERR_NOMEM";
    case CT_ERR_CUDA: return "CT_ERR_CUDA";
    case CT_ERR_RANK: return "CT_ERR_RANK";
    case CT_ERR_NONFINITE: return "CT_ERR_NONFINITE";
    case CT_ERR_NOCONVERGE: return "CT_ERR_NOCONVERGE";
    case CT_ERR_TIMEOUT: return "CT_ERR_TIMEOUT";
    case CT_ERR_UNSUPPORTED: return "CT_ERR_UNSUPPORTED";
  }
  return "CT_ERR_UNKNOWN";
}

const char* ct_version(void) { return "ctqr 0.1 (sm_103a)"; }

ct_status ct_system_size(const ct_geometry* g, double lambda, int64_t* m, int64_t* n) {
  if (!geometry_ok(g) || !(lambda >= 0.0) || !isfinite(lambda)) return CT_ERR_INVALID;
  const int64_t nn = (int64_t)g->nx * g->ny;
  const int64_t mm = (int64_t)g->n_views * g->n_bins + (lambda > 0.0 ? nn : 0);
  if (m) *m = mm;
  if (n) *n = nn;
  return CT_OK;
}

ct_status ct_build_system(const ct_geometry* g, ct_dtype dtype, double lambda, void* A,
                          int64_t lda, void* stream) {
  int64_t m = 0, n = 0;
  ct_status st = ct_system_size(g, lambda, &m, &n);
  if (st != CT_OK) return st;
  if (!A || !aligned16(A) || lda < m || (dtype != CT_F64 && dtype != CT_F32)) return CT_ERR_INVALID;
  return launch_build_system(g, dtype, lambda, A, lda, m, n, as_stream(stream));
}

ct_status ct_qr_factor(const void* A, ct_dtype dtype, int64_t m, int64_t n, int64_t lda,
                       ct_prec prec, const ct_qr_opts* opts, ct_factor** out, void* stream) {
  if (!out) return CT_ERR_INVALID;
  *out = nullptr;
  if (!A || !aligned16(A) || n < 1 || m < n || lda < m) return CT_ERR_INVALID;
  if (dtype != CT_F64 && dtype != CT_F32) return CT_ERR_INVALID;
  if (prec != CT_PREC_F64 && prec != CT_PREC_F32 && !tc_prec(prec)) return CT_ERR_INVALID;
  const ct_dtype store = prec == CT_PREC_F64 ? CT_F64 : CT_F32;
  const bool in_place = opts && opts->in_place;
  if (in_place && dtype != store) return CT_ERR_INVALID;
  if (opts && (opts->nb < 0 || opts->nb > 64)) return CT_ERR_INVALID;
  cudaStream_t s = as_stream(stream);
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;

  ct_factor* f = new ct_factor;
  f->m = m;
  f->n = n;
  f->prec = prec;
  f->store = store;
  f->device = di.device;
  const bool tc = tc_prec(prec);
  const bool f16 = prec == CT_PREC_F16X3;
  const int passes = opts && opts->tf32_passes ? opts->tf32_passes : 3;
  if (tc && passes != 1 && passes != 3) { delete f; return CT_ERR_INVALID; }
  if (f16 && opts && opts->tf32_passes) { delete f; return CT_ERR_INVALID; }
  int outer = opts && opts->outer_nb ? opts->outer_nb : 256;
  if (outer != 128 && outer != 256) { delete f; return CT_ERR_INVALID; }
  if (prec == CT_PREC_F64 && outer == 256 && opts && opts->outer_nb) { delete f; return CT_ERR_INVALID; }
  int want = (opts && opts->nb) ? opts->nb : (prec == CT_PREC_F64 ? 64 : 32);
  // TF32 factors whose widths the caller leaves open take the tuned pair
  if (tc && !(opts && opts->nb) && !(opts && opts->outer_nb)) {
    if ((st = tuned_factor_widths(m, n, passes, prec, s, &want, &outer)) != CT_OK) { delete f; return st; }
  }
  if (tc && (want > 32 || (want & (want - 1)))) { delete f; return CT_ERR_INVALID; }
  f->nb = panel_width_that_fits(m, want, di, store == CT_F64 ? 8 : 4, tc);
  const size_t es = elem_size(store);
  if (in_place) {
    f->F = (void*)A;
    f->owns_F = false;
    f->ld = lda;
  } else {
    f->ld = (m + 3) / 4 * 4;  // 16-byte aligned columns for both element types
    st = dev_alloc((char**)&f->F, (size_t)f->ld * n * es);
    if (st != CT_OK) { free_factor(f); return st; }
  }
  const int64_t np = ctqr::npanels(f);
  if ((st = alloc_factor_aux(f, di)) != CT_OK) {
    free_factor(f);
    return st;
  }
  cudaError_t ce = cudaMemsetAsync(f->status, 0, sizeof(int), s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(f->T, 0, (size_t)np * f->nb * f->nb * sizeof(double), s);
  if (ce != cudaSuccess) { free_factor(f); return CT_ERR_CUDA; }
  if (!in_place) {
    st = launch_copy_matrix(A, dtype, lda, f->F, store, f->ld, m, n, s);
    if (st != CT_OK) { free_factor(f); return st; }
  }
  const size_t work_elems = reflector_work_elems(di.sms, f->nb, n);
  Scratch work;
  if ((st = work.alloc(work_elems * sizeof(double), s)) != CT_OK) { free_factor(f); return st; }
  // One panel (factor + update of the columns [j0+nbp, cend) to its right).
  auto panel_step = [&](int64_t j0, int nbp, int64_t cend) -> ct_status {
    double* Tp = f->T + (size_t)(j0 / f->nb) * f->nb * f->nb;
    ct_status r = launch_panel(f, j0, nbp, Tp, s);
    if (r != CT_OK || j0 + nbp >= cend) return r;
    ReflectorArgs a;
    a.V = (const char*)f->F + (size_t)(j0 + j0 * f->ld) * es;
    a.v_f64 = store == CT_F64;
    a.ldv = f->ld;
    a.T = Tp;
    a.ldt = f->nb;
    a.nbp = nbp;
    a.C = (char*)f->F + (size_t)(j0 + (j0 + nbp) * f->ld) * es;
    a.c_f64 = store == CT_F64;
    a.ldc = f->ld;
    a.mr = m - j0;
    a.nc = cend - j0 - nbp;
    a.fp32_math = store == CT_F32;
    // two-level factors: the inner panels' updates in one launch when they fit
    if (tc && f->panel_cap == 0) {
      const ct_status u = inner_update_persist(f, j0, nbp, cend, Tp, (double*)work.p, work_elems, di.sms, s);
      if (u != CT_ERR_UNSUPPORTED) return u;
    }
    return apply_block_reflector(a, (double*)work.p, work_elems, di.sms, s);
  };
  // FP64 factors whose panels had to be narrowed for a tall matrix (or on
  // request, outer_nb = 128) update the trailing matrix once per outer block
  // of 128 // nb panels instead of once per panel
  const int outer_req = opts ? opts->outer_nb : 0;
  const bool two_level64 = store == CT_F64 && n > 128 && (outer_req == 128 || (outer_req == 0 && f->nb < 64));
  if (!tc && two_level64) {
    const int ow = (128 / f->nb) * f->nb;
    const size_t w64 = fp64_outer_work_elems(di.sms, n);
    Scratch ow64;
    if ((st = ow64.alloc(w64 * sizeof(double), s)) != CT_OK) { free_factor(f); return st; }
    for (int64_t J = 0; J < n; J += ow) {
      const int nbo = (int)(n - J < ow ? n - J : ow);
      for (int64_t j0 = J; j0 < J + nbo; j0 += f->nb) {
        const int nbp = (int)(J + nbo - j0 < f->nb ? J + nbo - j0 : f->nb);
        if ((st = panel_step(j0, nbp, J + nbo)) != CT_OK) { free_factor(f); return st; }
      }
      if ((st = fp64_outer_update(f, J, nbo, (double*)ow64.p, w64, di.sms, s)) != CT_OK) { free_factor(f); return st; }
    }
  } else if (!tc) {
    for (int64_t j0 = 0; j0 < n; j0 += f->nb) {
      const int nbp = (int)(n - j0 < f->nb ? n - j0 : f->nb);
      if ((st = panel_step(j0, nbp, n)) != CT_OK) { free_factor(f); return st; }
    }
  } else {
    // Outer blocks of 256 columns (or 128): inner panels update only their
    // own 128-column half, the first half's block reflector updates the
    // second half, and the rest of the matrix gets one tensor-core update
    // per outer block.
    const size_t owf = f16 ? outer_work_floats16(di.sms, m, n, outer) : outer_work_floats(di.sms, m, n, outer);
    Scratch owork, cwork;
    if ((st = owork.alloc(owf * sizeof(float), s)) != CT_OK) { free_factor(f); return st; }
    // FP16-split updates: bounds on the trailing columns' magnitudes (the
    // first block's from one pass over the matrix)
    F16Cols cols;
    if (f16) {
      if ((st = cwork.alloc((size_t)n * (sizeof(double) + sizeof(unsigned)), s)) != CT_OK) {
        free_factor(f);
        return st;
      }
      cols.acc = (double*)cwork.p;
      cols.bound = (unsigned*)(cols.acc + n);
      if ((st = f16_bounds(f, &cols, s)) != CT_OK) {
        free_factor(f);
        return st;
      }
    }
    // Look-ahead (opt-in, CTQR_LOOKAHEAD=1): while the columns beyond the
    // next outer block are updated on a second stream (on all but kReserve
    // SMs), the next block's panels and inner updates run on the reserved
    // SMs, when those panels fit on kReserve CTAs.  Measured on the 128x128
    // fan-beam system it is slower (the panels on 24 CTAs beside the
    // bandwidth-bound update take 425 instead of 150 us), so it is off by
    // default.  The guard below makes s wait for a deferred update on every
    // exit, before owork is released.
    constexpr int kReserve = 24;
    Lookahead la;
    la.reserve = kReserve;
    struct LaGuard {
      Lookahead* la;
      cudaStream_t s;
      ~LaGuard() {
        if (la->rest_pending) cudaStreamWaitEvent(s, la->ev_rest, 0);
        if (la->ev_t) cudaStreamWaitEvent(s, la->ev_t, 0);  // the last T on the side stream
        if (la->ev_w) cudaEventDestroy(la->ev_w);
        if (la->ev_rest) cudaEventDestroy(la->ev_rest);
        if (la->s2) cudaStreamDestroy(la->s2);
        if (la->ev_g) cudaEventDestroy(la->ev_g);
        if (la->ev_t) cudaEventDestroy(la->ev_t);
        if (la->s3) cudaStreamDestroy(la->s3);
      }
    } la_guard{&la, s};
    // the side stream for each outer block's T (beside its V^T C product)
    if (cudaStreamCreateWithFlags(&la.s3, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&la.ev_g, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&la.ev_t, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      free_factor(f);
      return CT_ERR_CUDA;
    }
    const char* la_env = getenv("CTQR_LOOKAHEAD");
    const bool la_on = !f16 && outer == 128 && la_env && *la_env == '1' && di.sms > 2 * kReserve;
    if (la_on) {
      if (cudaStreamCreateWithFlags(&la.s2, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&la.ev_w, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&la.ev_rest, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_factor(f);
        return CT_ERR_CUDA;
      }
    }
    auto half_panels = [&](int64_t J0, int nbo) -> ct_status {
      for (int64_t j0 = J0; j0 < J0 + nbo; j0 += f->nb) {
        const int nbp = (int)(J0 + nbo - j0 < f->nb ? J0 + nbo - j0 : f->nb);
        ct_status r = panel_step(j0, nbp, J0 + nbo);
        if (r != CT_OK) return r;
      }
      return CT_OK;
    };
    for (int64_t J = 0; outer == 256 && J < n; J += 256) {
      const int nbo_a = (int)(n - J < 128 ? n - J : 128);
      const int nbo_b = (int)(n - J - 128 <= 0 ? 0 : (n - J - 128 < 128 ? n - J - 128 : 128));
      if ((st = half_panels(J, nbo_a)) != CT_OK) { free_factor(f); return st; }
      if (nbo_b == 0) break;
      if ((st = f16 ? outer_update16(f, J, nbo_a, (float*)owork.p, owf, di.sms, s, &la, J + 128 + nbo_b, &cols)
                    : outer_block_update(f, J, nbo_a, (float*)owork.p, owf, di.sms, passes == 3, s, &la,
                                         J + 128 + nbo_b)) != CT_OK ||
          (st = half_panels(J + 128, nbo_b)) != CT_OK ||
          (st = f16 ? outer_update256_16(f, J, nbo_b, (float*)owork.p, owf, di.sms, s, &la, &cols)
                    : outer_block_update256(f, J, nbo_b, (float*)owork.p, owf, di.sms, passes == 3, s, &la)) !=
              CT_OK) {
        free_factor(f);
        return st;
      }
    }
    for (int64_t J = 0; outer == 128 && J < n; J += 128) {
      const int nbo = (int)(n - J < 128 ? n - J : 128);
      // this block's panels run beside the previous block's deferred update
      f->panel_cap = la.rest_pending ? kReserve : 0;
      for (int64_t j0 = J; j0 < J + nbo; j0 += f->nb) {
        const int nbp = (int)(J + nbo - j0 < f->nb ? J + nbo - j0 : f->nb);
        if ((st = panel_step(j0, nbp, J + nbo)) != CT_OK) { free_factor(f); return st; }
      }
      f->panel_cap = 0;
      la.defer = la_on && J + 256 < n && panel_fits_ctas(m - (J + 128), f->nb, kReserve, di);
      if ((st = f16 ? outer_update16(f, J, nbo, (float*)owork.p, owf, di.sms, s, &la, 0, &cols)
                    : outer_block_update(f, J, nbo, (float*)owork.p, owf, di.sms, passes == 3, s, &la)) != CT_OK) {
        free_factor(f);
        return st;
      }
    }
    if (la.rest_pending) {
      CT_CUDA_TRY(cudaStreamWaitEvent(s, la.ev_rest, 0));
      la.rest_pending = false;
    }
  }
  st = launch_rank_check(f, s);
  if (st != CT_OK) { free_factor(f); return st; }
  *out = f;
  return CT_OK;
}

ct_status ct_factor_info(const ct_factor* f, int64_t* m, int64_t* n, int* nb, ct_prec* prec) {
  if (!f) return CT_ERR_INVALID;
  if (m) *m = f->m;
  if (n) *n = f->n;
  if (nb) *nb = f->nb;
  if (prec) *prec = f->prec;
  return CT_OK;
}

ct_status ct_factor_data(const ct_factor* f, const void** F, ct_dtype* dtype, int64_t* ld,
                         const double** tau) {
  if (!f) return CT_ERR_INVALID;
  if (F) *F = f->F;
  if (dtype) *dtype = f->store;
  if (ld) *ld = f->ld;
  if (tau) *tau = f->tau;
  return CT_OK;
}

ct_status ct_factor_copy(const ct_factor* f, void* F_out, int64_t ld_out, double* tau_out,
                         void* stream) {
  if (!f) return CT_ERR_INVALID;
  cudaStream_t s = as_stream(stream);
  if (F_out && f->F_host) {  // the host factor's matrix, copied up to HBM
    if (ld_out < f->m) return CT_ERR_INVALID;
    CT_CUDA_TRY(cudaMemcpy2DAsync(F_out, ld_out * sizeof(double), f->F, f->ld * sizeof(double),
                                  f->m * sizeof(double), f->n, cudaMemcpyHostToDevice, s));
    F_out = nullptr;
  }
  if (F_out) {
    if (ld_out < f->m) return CT_ERR_INVALID;
    ct_status st = launch_copy_matrix(f->F, f->store, f->ld, F_out, f->store, ld_out, f->m, f->n, s);
    if (st != CT_OK) return st;
  }
  if (tau_out)
    CT_CUDA_TRY(cudaMemcpyAsync(tau_out, f->tau, sizeof(double) * f->n, cudaMemcpyDeviceToDevice, s));
  return CT_OK;
}

ct_status ct_factor_status(const ct_factor* f, void* stream) {
  if (!f) return CT_ERR_INVALID;
  return read_status(f, as_stream(stream));
}

ct_status ct_apply_qt(const ct_factor* f, double* B, int64_t ldb, int64_t k, void* stream) {
  if (!f || k < 0) return CT_ERR_INVALID;
  if (k == 0) return CT_OK;
  if (!B || !aligned16(B) || ldb < f->m) return CT_ERR_INVALID;
  cudaStream_t s = as_stream(stream);
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  const size_t work_elems = reflector_work_elems(di.sms, f->nb, k);
  Scratch work;
  if ((st = work.alloc(work_elems * sizeof(double), s)) != CT_OK) return st;
  return apply_qt_all(f, B, true, ldb, k, false, (double*)work.p, work_elems, di.sms, s);
}

ct_status ct_apply_qt_f32(const ct_factor* f, float* B, int64_t ldb, int64_t k, void* stream) {
  if (!f || k < 0) return CT_ERR_INVALID;
  if (f->store != CT_F32) return CT_ERR_UNSUPPORTED;
  if (k == 0) return CT_OK;
  if (!B || !aligned16(B) || ldb < f->m) return CT_ERR_INVALID;
  cudaStream_t s = as_stream(stream);
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  const size_t work_elems = reflector_work_elems(di.sms, f->nb, k);
  Scratch work;
  if ((st = work.alloc(work_elems * sizeof(double), s)) != CT_OK) return st;
  return apply_qt_all(f, B, false, ldb, k, true, (double*)work.p, work_elems, di.sms, s);
}

ct_status ct_trsm_solve(const ct_factor* f, double* B, int64_t ldb, int64_t k, void* stream) {
  if (!f || k < 0) return CT_ERR_INVALID;
  if (k == 0) return CT_OK;
  if (!B || !aligned16(B) || ldb < f->n) return CT_ERR_INVALID;
  return launch_trsm(f, B, true, ldb, k, as_stream(stream));
}

ct_status ct_trsm_solve_f32(const ct_factor* f, float* B, int64_t ldb, int64_t k, int transpose, void* stream) {
  if (!f || k < 0) return CT_ERR_INVALID;
  if (f->store != CT_F32) return CT_ERR_UNSUPPORTED;
  if (k == 0) return CT_OK;
  if (!B || !aligned16(B) || ldb < f->n) return CT_ERR_INVALID;
  cudaStream_t s = as_stream(stream);
  return transpose ? launch_trsm_t(f, B, false, ldb, k, s) : launch_trsm(f, B, false, ldb, k, s);
}

static ct_status reconstruct_impl(const ct_factor* f, const void* A, ct_dtype A_dtype, int64_t lda,
                                  const SparseSystem* sp, const double* B, int64_t ldb, double* X, int64_t ldx,
                                  int64_t k, const ct_refine_opts* ropts, ct_report* report, void* stream);

ct_status ct_reconstruct_batch(const ct_factor* f, const void* A, ct_dtype A_dtype, int64_t lda,
                               const double* B, int64_t ldb, double* X, int64_t ldx, int64_t k,
                               const ct_refine_opts* ropts, ct_report* report, void* stream) {
  return reconstruct_impl(f, A, A_dtype, lda, nullptr, B, ldb, X, ldx, k, ropts, report, stream);
}

static ct_status reconstruct_impl(const ct_factor* f, const void* A, ct_dtype A_dtype, int64_t lda,
                                  const SparseSystem* sp, const double* B, int64_t ldb, double* X, int64_t ldx,
                                  int64_t k, const ct_refine_opts* ropts, ct_report* report, void* stream) {
  const auto t_start = std::chrono::steady_clock::now();
  if (report) memset(report, 0, sizeof(*report));
  if (!f || k < 0) return CT_ERR_INVALID;
  if (k == 0) return CT_OK;
  if (!B || !X || !aligned16(B) || !aligned16(X) || ldb < f->m || ldx < f->n) return CT_ERR_INVALID;
  const int64_t a_rows = (ropts && ropts->lambda > 0.0) ? f->m - f->n : f->m;
  if (A && (!aligned16(A) || lda < a_rows || (A_dtype != CT_F64 && A_dtype != CT_F32))) return CT_ERR_INVALID;
  cudaStream_t s = as_stream(stream);
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  const int64_t m = f->m, n = f->n;

  if (!A && !sp) {
    const int64_t ldw = (m + 3) / 4 * 4;
    const size_t work_elems = reflector_work_elems(di.sms, f->nb, k);
    Scratch work, Y;
    if ((st = work.alloc(work_elems * sizeof(double), s)) != CT_OK) return st;
    if ((st = Y.alloc((size_t)ldw * k * sizeof(double), s)) != CT_OK) return st;
    double* Yd = (double*)Y.p;
    // Plain solve in FP64 arithmetic: Y = B; Y = Q^T Y; Y[0:n] = R^-1 Y[0:n]; X = Y[0:n].
    if ((st = launch_copy_matrix(B, CT_F64, ldb, Yd, CT_F64, ldw, m, k, s)) != CT_OK) return st;
    if ((st = apply_qt_all(f, Yd, true, ldw, k, false, (double*)work.p, work_elems, di.sms, s)) != CT_OK) return st;
    if ((st = launch_trsm(f, Yd, true, ldw, k, s)) != CT_OK) return st;
    if ((st = launch_copy_matrix(Yd, CT_F64, ldw, X, CT_F64, ldx, n, k, s)) != CT_OK) return st;
    st = read_status(f, s);
    if (report) report->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return st;
  }

  Refiner R(f, A, A_dtype, lda, sp, B, ldb, X, ldx, k, s, di.sms);
  st = R.run(ropts, report);
  ct_status dev = read_status(f, s);
  if (report) report->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (dev != CT_OK) return dev;
  return st;
}

}  // extern "C"

namespace ctqr {
ct_status reconstruct_with(const ct_factor* f, const SparseSystem* sp, const double* B, int64_t ldb, double* X,
                           int64_t ldx, int64_t k, const ct_refine_opts* ropts, ct_report* report, cudaStream_t s) {
  return reconstruct_impl(f, nullptr, CT_F64, 0, sp, B, ldb, X, ldx, k, ropts, report, (void*)s);
}
}  // namespace ctqr

extern "C" {

ct_status ct_reconstruct_scan(const ct_geometry* geom, double lambda, ct_prec prec,
                              const double* B, int64_t ldb, double* X, int64_t ldx, int64_t k,
                              ct_buffers where, const ct_refine_opts* ropts, ct_report* report,
                              void* stream) {
  const auto t_start = std::chrono::steady_clock::now();
  if (report) memset(report, 0, sizeof(*report));
  int64_t m = 0, n = 0;
  ct_status st = ct_system_size(geom, lambda, &m, &n);
  if (st != CT_OK) return st;
  if (k < 0 || (k > 0 && (!B || !X || ldb < m || ldx < n))) return CT_ERR_INVALID;
  if (where != CT_DEVICE_BUFFERS && where != CT_HOST_BUFFERS) return CT_ERR_INVALID;
  if (prec != CT_PREC_F64 && prec != CT_PREC_F32 && !tc_prec(prec)) return CT_ERR_INVALID;
  if (m < n) return CT_ERR_INVALID;
  if (k == 0) return CT_OK;
  cudaStream_t s = as_stream(stream);
  const bool host = where == CT_HOST_BUFFERS;
  if (!host && (!aligned16(B) || !aligned16(X))) return CT_ERR_INVALID;
  const int64_t lda = (m + 3) / 4 * 4;
  const bool mixed = prec != CT_PREC_F64;
  Scratch Abuf, Bbuf, Xbuf;
  // FP64: [A; lambda I] in FP64, factored in place.  Mixed: [A; lambda I] in
  // FP32, factored in place, plus the exact sparse FP64 A for the residuals.
  if ((st = Abuf.alloc((size_t)lda * n * (mixed ? sizeof(float) : sizeof(double)), s)) != CT_OK) return st;
  const double* Bd = B;
  double* Xd = X;
  int64_t ldbd = ldb, ldxd = ldx;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  for (auto& e : ev) CT_CUDA_TRY(cudaEventCreate(&e));
  struct EvFree {
    cudaEvent_t* e;
    ~EvFree() { for (int i = 0; i < 4; ++i) if (e[i]) cudaEventDestroy(e[i]); }
  } evfree{ev};
  if (host) {
    if ((st = Bbuf.alloc((size_t)lda * k * sizeof(double), s)) != CT_OK) return st;
    if ((st = Xbuf.alloc((size_t)n * k * sizeof(double), s)) != CT_OK) return st;
    CT_CUDA_TRY(cudaMemcpy2DAsync(Bbuf.p, lda * sizeof(double), B, ldb * sizeof(double),
                                  m * sizeof(double), k, cudaMemcpyHostToDevice, s));
    Bd = (const double*)Bbuf.p;
    Xd = (double*)Xbuf.p;
    ldbd = lda;
    ldxd = n;
  }
  int* sp_status = nullptr;
  CT_CUDA_TRY(cudaMallocAsync((void**)&sp_status, sizeof(int), s));
  struct SFree { int* p; cudaStream_t s; ~SFree() { cudaFreeAsync(p, s); } } sfree{sp_status, s};
  CT_CUDA_TRY(cudaMemsetAsync(sp_status, 0, sizeof(int), s));
  SparseSystem sp;
  CT_CUDA_TRY(cudaEventRecord(ev[0], s));
  if ((st = launch_build_system(geom, mixed ? CT_F32 : CT_F64, lambda, Abuf.p, lda, m, n, s)) != CT_OK) return st;
  if (mixed && (st = sp.build(geom, k, sp_status, s)) != CT_OK) return st;
  CT_CUDA_TRY(cudaEventRecord(ev[1], s));
  ct_factor* f = nullptr;
  ct_qr_opts qo = {0, 1, 0, 0};  // factor in place
  if ((st = ct_qr_factor(Abuf.p, mixed ? CT_F32 : CT_F64, m, n, lda, prec, &qo, &f, stream)) != CT_OK) return st;
  CT_CUDA_TRY(cudaEventRecord(ev[2], s));
  ct_refine_opts ro = ropts ? *ropts : ct_refine_opts{0, 0.0, 0.0, 0};
  ro.lambda = lambda;
  ct_report rep;
  ct_status rs = reconstruct_impl(f, nullptr, CT_F64, 0, mixed ? &sp : nullptr, Bd, ldbd, Xd, ldxd, k, &ro, &rep,
                                  stream);
  if (rs == CT_OK && mixed) {
    int h = 0;
    if (cudaMemcpyAsync(&h, sp_status, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess && h != 0)
      rs = (ct_status)h;
  }
  cudaError_t ce = cudaEventRecord(ev[3], s);
  if (ce == cudaSuccess && host)
    ce = cudaMemcpy2DAsync(X, ldx * sizeof(double), Xd, ldxd * sizeof(double), n * sizeof(double), k,
                           cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  ct_factor_destroy(f);
  if (ce != cudaSuccess) return CT_ERR_CUDA;
  if (report) {
    *report = rep;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ev[0], ev[1]) == cudaSuccess) report->ms_build = t;
    if (cudaEventElapsedTime(&t, ev[1], ev[2]) == cudaSuccess) report->ms_factor = t;
    if (cudaEventElapsedTime(&t, ev[2], ev[3]) == cudaSuccess) report->ms_solve = t;
    report->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  }
  return rs;
}

static int* gemm_status_word(ct_status* err) {
  static int* word = nullptr;
  if (!word) {
    if (cudaMalloc((void**)&word, sizeof(int)) != cudaSuccess || cudaMemset(word, 0, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      word = nullptr;
      *err = CT_ERR_NOMEM;
    }
  }
  return word;
}

ct_status ct_gemm_tf32_tn(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                          int64_t ldb, float* C, int64_t ldc, int accumulate, int split3, void* stream) {
  if (M < 0 || N < 0 || K < 0) return CT_ERR_INVALID;
  if (M == 0 || N == 0) return CT_OK;
  ct_status err = CT_OK;
  int* status = gemm_status_word(&err);
  if (!status) return err;
  return tc_gemm_tn(A, lda, B, ldb, M, N, K, C, ldc, 0, accumulate ? 1 : 0, 1, split3 != 0, status,
                    as_stream(stream));
}

ct_status ct_gemm_f16x3_tn(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B,
                           int64_t ldb, float* C, int64_t ldc, int accumulate, void* stream) {
  if (M < 0 || N < 0 || K < 0) return CT_ERR_INVALID;
  if (M == 0 || N == 0) return CT_OK;
  if (!A || !B || !C || !aligned16(A) || !aligned16(B) || lda < K || ldb < K || ldc < M || (lda & 3) || (ldb & 3))
    return CT_ERR_INVALID;
  if (M > 65535 || N > 65535 || (accumulate && K > 256)) return CT_ERR_INVALID;
  ct_status err = CT_OK;
  int* status = gemm_status_word(&err);
  if (!status) return err;
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  cudaStream_t s = as_stream(stream);
  if (K == 0) {
    if (accumulate) return CT_OK;
    return launch_zero_matrix(C, sizeof(float), ldc, M, N, s);
  }
  const int64_t ldk = (K + 7) / 8 * 8;
  const size_t ha = (size_t)ldk * M, hb = (size_t)ldk * N;
  Scratch work;
  if ((st = work.alloc((2 * ha + 2 * hb) * sizeof(__half) + (size_t)N * 16 + 1024, s)) != CT_OK) return st;
  __half* Ah = (__half*)work.p;
  __half* Al = Ah + ha;
  __half* Bh = Al + ha;
  __half* Bl = Bh + hb;
  unsigned* bmax = (unsigned*)(((uintptr_t)(Bl + hb) + 15) & ~(uintptr_t)15);
  // colinv: 16-byte aligned, readable up to N rounded up to 128 entries
  float* colinv = (float*)(((uintptr_t)(bmax + N) + 15) & ~(uintptr_t)15);
  double* nacc = (double*)(((uintptr_t)(colinv + N + 128) + 15) & ~(uintptr_t)15);
  if ((st = launch_split16(A, lda, K, M, nullptr, 8, 0, Ah, Al, ldk, nullptr, s)) != CT_OK) return st;
  if ((st = launch_colnorm_bound(B, ldb, K, N, nacc, bmax, s)) != CT_OK) return st;
  if (!accumulate)
    return tc_gemm16(Ah, Al, ldk, B, nullptr, ldb, bmax, nullptr, M, N, K, 1.f / 256.f, C, ldc, 0, 1, status, s,
                     nullptr);
  if ((st = launch_split16(B, ldb, K, N, bmax, 0, 8, Bh, Bl, ldk, colinv, s)) != CT_OK) return st;
  return tc_update16(Ah, Al, ldk, Bh, Bl, ldk, colinv, M, N, K, C, ldc, di.sms, status, s);
}

ct_status ct_gemm_status(void* stream) {
  ct_status err = CT_OK;
  int* status = gemm_status_word(&err);
  if (!status) return err;
  int h = 0;
  cudaStream_t s = as_stream(stream);
  CT_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CT_CUDA_TRY(cudaStreamSynchronize(s));
  if (h != 0) CT_CUDA_TRY(cudaMemset(status, 0, sizeof(int)));
  return (ct_status)h;
}

ct_status ct_qr_solve_batched(int count, const ct_batch_system* systems, const ct_batch_opts* opts,
                              ct_batch_report* report, void* stream) {
  if (report) memset(report, 0, sizeof(*report));
  if (count < 0 || (count > 0 && !systems)) return CT_ERR_INVALID;
  if (count == 0) return CT_OK;
  int64_t med_m = 0, med_n = 0;
  std::vector<std::pair<int64_t, int64_t>> sizes;
  for (int i = 0; i < count; ++i) {
    const ct_batch_system& q = systems[i];
    if (q.n < 1 || q.m < q.n || !q.A || q.lda < q.m || q.k < 0 || (q.k > 0 && (!q.B || q.ldb < q.m)))
      return CT_ERR_INVALID;
    sizes.push_back({q.n, q.m});
  }
  std::sort(sizes.begin(), sizes.end());
  med_n = sizes[count / 2].first;
  med_m = sizes[count / 2].second;
  cudaStream_t s = as_stream(stream);
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  const int bprec = opts ? opts->prec : CT_PREC_F64;
  if (bprec != CT_PREC_F64 && !tc_prec((ct_prec)bprec)) return CT_ERR_INVALID;
  if (tc_prec((ct_prec)bprec)) {
    // one system after another through the tensor-core factorization and
    // the FP64 refinement against its own (unchanged) FP64 A
    const auto t0 = std::chrono::steady_clock::now();
    int worst_it = 0;
    ct_status agg = CT_OK;
    for (int i = 0; i < count; ++i) {
      const ct_batch_system& q = systems[i];
      ct_factor* f = nullptr;
      if ((st = ct_qr_factor(q.A, CT_F64, q.m, q.n, q.lda, (ct_prec)bprec, nullptr, &f, stream)) != CT_OK) return st;
      if (q.k > 0) {
        Scratch xs;
        if ((st = xs.alloc((size_t)q.n * q.k * sizeof(double), s)) != CT_OK) {
          ct_factor_destroy(f);
          return st;
        }
        ct_report rep;
        ct_status rs = ct_reconstruct_batch(f, q.A, CT_F64, q.lda, q.B, q.ldb, (double*)xs.p, q.n, q.k, nullptr,
                                            &rep, stream);
        if (rep.iterations > worst_it) worst_it = rep.iterations;
        if (rs == CT_OK)
          rs = launch_copy_matrix(xs.p, CT_F64, q.n, q.B, CT_F64, q.ldb, q.n, q.k, s);
        if (rs != CT_OK && agg == CT_OK) agg = rs;
      } else {
        const ct_status fs = ct_factor_status(f, stream);
        if (fs != CT_OK && agg == CT_OK) agg = fs;
      }
      ct_factor_destroy(f);
    }
    CT_CUDA_TRY(cudaStreamSynchronize(s));
    if (report) {
      report->tile = 0;
      report->tasks = 0;
      report->iterations = worst_it;
      report->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    return agg;
  }
  int tile = opts ? opts->tile : 0;
  if (tile != 0 && tile != 32 && tile != 64) return CT_ERR_INVALID;
  // Large batches take the larger tile without measuring: the task list of
  // 32-wide tiles would exceed 2^25 tasks (~3.4 GB).
  if (tile == 0 && batch_task_count(count, systems, 32) > (int64_t(1) << 25)) tile = 64;
  if (tile == 0 && (st = tuned_batch_tile(med_m, med_n, di.sms, s, &tile)) != CT_OK) return st;
  if (batch_task_count(count, systems, tile) > INT32_MAX) return CT_ERR_UNSUPPORTED;
  int* status = nullptr;
  CT_CUDA_TRY(cudaMallocAsync((void**)&status, sizeof(int), s));
  struct F { int* p; cudaStream_t s; ~F() { cudaFreeAsync(p, s); } } fr{status, s};
  CT_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
  double ms = 0.0;
  int ntasks = 0;
  if ((st = run_batch(count, systems, tile, di.sms, status, s, !(opts && opts->no_cache), &ms, &ntasks)) != CT_OK)
    return st;
  // Rank test on every R (same threshold as ct_qr_factor).
  for (int i = 0; i < count; ++i) {
    ct_factor tmp;
    tmp.m = systems[i].m;
    tmp.n = systems[i].n;
    tmp.ld = systems[i].lda;
    tmp.store = CT_F64;
    tmp.F = systems[i].A;
    tmp.status = status;
    if ((st = launch_rank_check(&tmp, s)) != CT_OK) { tmp.F = nullptr; tmp.status = nullptr; return st; }
    tmp.F = nullptr;
    tmp.status = nullptr;
  }
  int h = 0;
  CT_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CT_CUDA_TRY(cudaStreamSynchronize(s));
  if (report) {
    report->tile = tile;
    report->ms = ms;
    report->tasks = ntasks;
  }
  return (ct_status)h;
}

void ct_qr_solve_batched_release(void) { release_batch_cache(); }

ct_status ct_batch_plan(int count, const ct_batch_system* systems, int tile, int32_t* tasks, int64_t max_tasks,
                        int64_t* ntasks, int* nparts) {
  if (count < 1 || !systems) return CT_ERR_INVALID;
  for (int i = 0; i < count; ++i) {
    const ct_batch_system& q = systems[i];
    if (q.n < 1 || q.m < q.n || q.lda < q.m || q.k < 0 || (q.k > 0 && q.ldb < q.m)) return CT_ERR_INVALID;
  }
  return export_batch_plan(count, systems, tile, tasks, max_tasks, ntasks, nparts);
}

void ct_factor_destroy(ct_factor* f) {
  if (!f) return;
  cudaDeviceSynchronize();
  free_factor(f);
}

}  // extern "C"
