// api.cu -- the C ABI of include/ctqr.h: argument checks, the factor's
// lifetime, and the host-side sequencing of the kernels on the caller's stream.
#include <math.h>
#include <stdlib.h>
#include <string.h>

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

void free_factor(ct_factor* f) {
  if (!f) return;
  if (f->owns_F && f->F) cudaFree(f->F);
  if (f->tau) cudaFree(f->tau);
  if (f->T) cudaFree(f->T);
  if (f->status) cudaFree(f->status);
  if (f->barrier) cudaFree(f->barrier);
  if (f->partials) cudaFree(f->partials);
  delete f;
}

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

// Apply Q^T (all panels, factorization order) to the mr = m rows of C (k
// columns, element type c_f64 ? FP64 : FP32).
ct_status apply_qt_all(const ct_factor* f, void* C, bool c_f64, int64_t ldc, int64_t k, bool fp32_math,
                       double* work, size_t work_elems, int sms, cudaStream_t s) {
  const size_t es = elem_size(f->store), cs = c_f64 ? 8 : 4;
  for (int64_t j0 = 0, p = 0; j0 < f->n; j0 += f->nb, ++p) {
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
    ct_status st = apply_block_reflector(a, work, work_elems, sms, s);
    if (st != CT_OK) return st;
  }
  return CT_OK;
}

ct_status read_status(const ct_factor* f, cudaStream_t s) {
  int h = 0;
  CT_CUDA_TRY(cudaMemcpyAsync(&h, f->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CT_CUDA_TRY(cudaStreamSynchronize(s));
  return (ct_status)h;
}

}  // namespace

namespace ctqr {
int64_t npanels(const ct_factor* f) { return (f->n + f->nb - 1) / f->nb; }
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
  if (prec != CT_PREC_F64 && prec != CT_PREC_F32 && prec != CT_PREC_TF32) return CT_ERR_INVALID;
  if (prec == CT_PREC_TF32) return CT_ERR_UNSUPPORTED;
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
  int want = (opts && opts->nb) ? opts->nb : (prec == CT_PREC_F64 ? 64 : 32);
  f->nb = panel_width_that_fits(m, want, di);
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
  f->partials_elems = panel_partials_elems(di.sms, f->nb);
  if ((st = dev_alloc(&f->tau, (size_t)n)) != CT_OK ||
      (st = dev_alloc(&f->T, (size_t)np * f->nb * f->nb)) != CT_OK ||
      (st = dev_alloc(&f->status, 1)) != CT_OK ||
      (st = dev_alloc(&f->barrier, 2)) != CT_OK ||
      (st = dev_alloc(&f->partials, f->partials_elems)) != CT_OK) {
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

  for (int64_t j0 = 0, p = 0; j0 < n; j0 += f->nb, ++p) {
    const int nbp = (int)(n - j0 < f->nb ? n - j0 : f->nb);
    double* Tp = f->T + (size_t)p * f->nb * f->nb;
    st = launch_panel(f, j0, nbp, Tp, s);
    if (st != CT_OK) { free_factor(f); return st; }
    if (j0 + nbp < n) {
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
      a.nc = n - j0 - nbp;
      a.fp32_math = store == CT_F32;
      st = apply_block_reflector(a, (double*)work.p, work_elems, di.sms, s);
      if (st != CT_OK) { free_factor(f); return st; }
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

ct_status ct_trsm_solve(const ct_factor* f, double* B, int64_t ldb, int64_t k, void* stream) {
  if (!f || k < 0) return CT_ERR_INVALID;
  if (k == 0) return CT_OK;
  if (!B || !aligned16(B) || ldb < f->n) return CT_ERR_INVALID;
  return launch_trsm(f, B, true, ldb, k, as_stream(stream));
}

ct_status ct_reconstruct_batch(const ct_factor* f, const void* A, ct_dtype A_dtype, int64_t lda,
                               const double* B, int64_t ldb, double* X, int64_t ldx, int64_t k,
                               const ct_refine_opts* ropts, ct_report* report, void* stream) {
  const auto t_start = std::chrono::steady_clock::now();
  if (report) memset(report, 0, sizeof(*report));
  if (!f || k < 0) return CT_ERR_INVALID;
  if (k == 0) return CT_OK;
  if (!B || !X || !aligned16(B) || !aligned16(X) || ldb < f->m || ldx < f->n) return CT_ERR_INVALID;
  if (A && (!aligned16(A) || lda < f->m || (A_dtype != CT_F64 && A_dtype != CT_F32))) return CT_ERR_INVALID;
  const int max_iter = ropts && ropts->max_iter > 0 ? ropts->max_iter : 30;
  const double tol = ropts && ropts->tol > 0.0 ? ropts->tol : 1e-12;
  cudaStream_t s = as_stream(stream);
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  const int64_t m = f->m, n = f->n;
  const int64_t ldw = (m + 3) / 4 * 4;
  const size_t work_elems = reflector_work_elems(di.sms, f->nb, k);

  Scratch work, Y;
  if ((st = work.alloc(work_elems * sizeof(double), s)) != CT_OK) return st;
  if ((st = Y.alloc((size_t)ldw * k * sizeof(double), s)) != CT_OK) return st;
  double* Yd = (double*)Y.p;

  if (!A) {
    // Plain solve in FP64 arithmetic: Y = B; Y = Q^T Y; Y[0:n] = R^-1 Y[0:n]; X = Y[0:n].
    if ((st = launch_copy_matrix(B, CT_F64, ldb, Yd, CT_F64, ldw, m, k, s)) != CT_OK) return st;
    if ((st = apply_qt_all(f, Yd, true, ldw, k, false, (double*)work.p, work_elems, di.sms, s)) != CT_OK) return st;
    if ((st = launch_trsm(f, Yd, true, ldw, k, s)) != CT_OK) return st;
    if ((st = launch_copy_matrix(Yd, CT_F64, ldw, X, CT_F64, ldx, n, k, s)) != CT_OK) return st;
    st = read_status(f, s);
    if (report) report->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    return st;
  }

  // Refinement.  Corrections are solved in the factor's storage precision.
  const bool f32 = f->store == CT_F32;
  Scratch Dbuf, norms;
  if (f32 && (st = Dbuf.alloc((size_t)ldw * k * sizeof(float), s)) != CT_OK) return st;
  if ((st = norms.alloc((size_t)3 * k * sizeof(double), s)) != CT_OK) return st;
  double* dn2 = (double*)norms.p;
  double* xn2 = dn2 + k;
  double* bn2 = xn2 + k;
  std::vector<double> h(3 * (size_t)k);
  if ((st = launch_zero_matrix(X, 8, ldx, n, k, s)) != CT_OK) return st;
  if ((st = launch_col_norms2(B, ldb, m, k, bn2, s)) != CT_OK) return st;
  int it = 0;
  double last = INFINITY, resid = 0.0;
  ct_status result = CT_ERR_NOCONVERGE;
  for (; it <= max_iter; ++it) {
    // Res = B - A X (FP64); the first pass has X = 0, so Res = B.
    if ((st = launch_copy_matrix(B, CT_F64, ldb, Yd, CT_F64, ldw, m, k, s)) != CT_OK) return st;
    if (it > 0 && (st = launch_dense_update(A, A_dtype == CT_F64, lda, (int)n, X, ldx, Yd, true, ldw, m, k, s)) != CT_OK) return st;
    if (it > 0) {
      if ((st = launch_col_norms2(Yd, ldw, m, k, dn2, s)) != CT_OK) return st;
      CT_CUDA_TRY(cudaMemcpyAsync(h.data(), dn2, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
      CT_CUDA_TRY(cudaMemcpyAsync(h.data() + 2 * k, bn2, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
      CT_CUDA_TRY(cudaStreamSynchronize(s));
      double rr = 0.0, bb = 0.0;
      for (int64_t c = 0; c < k; ++c) { rr += h[c]; bb += h[2 * k + c]; }
      resid = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
    }
    if (f32) {
      float* D = (float*)Dbuf.p;
      if ((st = launch_copy_matrix(Yd, CT_F64, ldw, D, CT_F32, ldw, m, k, s)) != CT_OK) return st;
      if ((st = apply_qt_all(f, D, false, ldw, k, true, (double*)work.p, work_elems, di.sms, s)) != CT_OK) return st;
      if ((st = launch_trsm(f, D, false, ldw, k, s)) != CT_OK) return st;
      if ((st = launch_add_f32_to_f64(D, ldw, X, ldx, n, k, dn2, xn2, s)) != CT_OK) return st;
    } else {
      if ((st = apply_qt_all(f, Yd, true, ldw, k, false, (double*)work.p, work_elems, di.sms, s)) != CT_OK) return st;
      if ((st = launch_trsm(f, Yd, true, ldw, k, s)) != CT_OK) return st;
      if ((st = launch_add_f64_to_f64(Yd, ldw, X, ldx, n, k, dn2, xn2, s)) != CT_OK) return st;
    }
    CT_CUDA_TRY(cudaMemcpyAsync(h.data(), dn2, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost, s));
    CT_CUDA_TRY(cudaStreamSynchronize(s));
    double worst = 0.0;
    for (int64_t c = 0; c < k; ++c) {
      const double xc = sqrt(h[k + c]), dc = sqrt(h[c]);
      const double rel = xc > 0.0 ? dc / xc : (dc > 0.0 ? INFINITY : 0.0);
      if (!(rel <= worst)) worst = rel;
    }
    if (it > 0) last = worst;
    if (it > 0 && worst <= tol) { result = CT_OK; break; }
    if (!isfinite(worst)) { result = CT_ERR_NONFINITE; break; }
  }
  if (report) {
    report->iterations = it > max_iter ? max_iter : it;
    report->last_update = last;
    report->residual = resid;
  }
  ct_status dev = read_status(f, s);
  if (report) report->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (dev != CT_OK) return dev;
  return result;
}

void ct_factor_destroy(ct_factor* f) {
  if (!f) return;
  cudaDeviceSynchronize();
  free_factor(f);
}

}  // extern "C"
