// ooc.cu -- out-of-core factorization and solve: the matrix and its factor
// stay in host memory and stream through HBM block column by block column.
//
// This is the GPU form of the paper's out-of-core algorithm-by-blocks (Sec.
// II-B, II-C): there the matrix lives in tile files on disk, a block cache in
// RAM holds what the running tasks need, and an I/O thread reads ahead while
// the compute threads work (the O-OOC configuration of Sec. III; B-OOC without
// the overlap).  Here host memory plays the disk, HBM the cache, and a copy
// stream the I/O thread: while the compute stream applies or factors one block
// column, the copy stream brings the next one in (double buffering).
//
// Factorization, left-looking by block columns of width bw (a multiple of the
// panel width nb; the paper's left-looking order, Table tasks_qr_ab):
//   for each block column K:
//     A_K (all m rows) -> HBM
//     for each earlier block column I < K: V_I (rows I*bw..m) -> HBM (double
//       buffered) and A_K <- Q_I^T A_K, panel by panel (Apply_left_Qt_of_
//       dense_QR with the panel T factors, which stay in HBM)
//     factor A_K's rows K*bw..m in HBM (panels + their in-block updates)
//     A_K -> host (R above the diagonal, reflectors below)
// Solve: Q^T B streams every V_I once in factorization order; the back-solve
// streams R's block columns bottom-up (Trsm_lunn of the diagonal block, then
// the update of the rows above, Gemm_nn_mo).  B and X stay in HBM.
// FP64 throughout (the paper's arithmetic).  HBM holds three m x bw buffers.
#include <stdint.h>
#include <stdlib.h>

#include <vector>

#include "internal.cuh"

namespace ctqr {
namespace {

// A view of a device block column as a factor whose global column c0 is the
// buffer's first column: launch_panel and launch_trsm address F[j0 + j0*ld]
// with global indices.  The view's F is only ever offset by global indices
// >= c0, so every address formed lands inside the buffer.
ct_factor column_view(const ct_factor* f, double* buf, int64_t ldb, int64_t c0) {
  ct_factor v;
  v.m = f->m;
  v.n = f->n;
  v.ld = ldb;
  v.nb = f->nb;
  v.prec = CT_PREC_F64;
  v.store = CT_F64;
  v.F = (void*)((uintptr_t)buf - (uintptr_t)(c0 * ldb * sizeof(double)));
  v.owns_F = false;
  v.tau = f->tau;
  v.T = f->T;
  v.status = f->status;
  v.barrier = f->barrier;
  v.partials = f->partials;
  v.partials_elems = f->partials_elems;
  return v;
}

// diag[c0 + i] = A(c0 + i, i) for i < w: the block's R diagonal, kept in HBM
// for the rank test once all blocks are factored.
__global__ void k_block_diag(const double* __restrict__ A, int64_t ld, int64_t c0, int64_t w,
                             double* __restrict__ diag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < w) diag[c0 + i] = A[c0 + i + i * ld];
}

// Streams and events of one out-of-core pass (copy stream + two buffers).
struct Pipe {
  cudaStream_t cs = nullptr;
  cudaEvent_t loaded[2] = {nullptr, nullptr};  // buffer b holds its block (copy stream)
  cudaEvent_t freed[2] = {nullptr, nullptr};   // compute is done with buffer b
  cudaEvent_t start = nullptr;
  ct_status init(cudaStream_t s, bool overlap) {
    if (overlap) {
      CT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      CT_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
      CT_CUDA_TRY(cudaEventRecord(start, s));
      CT_CUDA_TRY(cudaStreamWaitEvent(cs, start, 0));  // copies follow the caller's earlier work
      for (int b = 0; b < 2; ++b) {
        CT_CUDA_TRY(cudaEventCreateWithFlags(&loaded[b], cudaEventDisableTiming));
        CT_CUDA_TRY(cudaEventCreateWithFlags(&freed[b], cudaEventDisableTiming));
      }
    }
    return CT_OK;
  }
  ~Pipe() {
    for (int b = 0; b < 2; ++b) {
      if (loaded[b]) cudaEventDestroy(loaded[b]);
      if (freed[b]) cudaEventDestroy(freed[b]);
    }
    if (start) cudaEventDestroy(start);
    if (cs) cudaStreamDestroy(cs);
  }
};

}  // namespace
}  // namespace ctqr

namespace ctqr {
namespace {

// Copy rows [r0, r1) of host block column [c0, c0 + w) to the device buffer
// (rows at their global offsets, ld ldd) or back.
ct_status copy_rows(const ct_factor* f, double* dev, int64_t ldd, int64_t r0, int64_t r1, int64_t c0, int64_t w,
                    bool to_dev, cudaStream_t cs) {
  if (r1 <= r0 || w <= 0) return CT_OK;
  double* host = (double*)f->F + r0 + c0 * f->ld;
  const size_t rows = (size_t)(r1 - r0);
  if (to_dev)
    CT_CUDA_TRY(cudaMemcpy2DAsync(dev + r0, ldd * sizeof(double), host, f->ld * sizeof(double),
                                  rows * sizeof(double), (size_t)w, cudaMemcpyHostToDevice, cs));
  else
    CT_CUDA_TRY(cudaMemcpy2DAsync(host, f->ld * sizeof(double), dev + r0, ldd * sizeof(double),
                                  rows * sizeof(double), (size_t)w, cudaMemcpyDeviceToHost, cs));
  return CT_OK;
}

// Stream the block columns seq[0], seq[1], ... through the two buffers: the
// copy stream loads block seq[t+1] while the compute stream `s` uses block
// seq[t] (with overlap; otherwise both happen on s, one after the other).
// load(I, buf, stream) issues the copy of block I; use(I, buf) the compute.
template <typename Load, typename Use>
ct_status stream_blocks(const int64_t* seq, int64_t count, double* const buf[2], Pipe& p, bool overlap,
                        cudaStream_t s, Load load, Use use) {
  if (count <= 0) return CT_OK;
  ct_status st;
  if (!overlap) {
    for (int64_t t = 0; t < count; ++t) {
      if ((st = load(seq[t], buf[0], s)) != CT_OK) return st;
      if ((st = use(seq[t], buf[0])) != CT_OK) return st;
    }
    return CT_OK;
  }
  if ((st = load(seq[0], buf[0], p.cs)) != CT_OK) return st;
  CT_CUDA_TRY(cudaEventRecord(p.loaded[0], p.cs));
  for (int64_t t = 0; t < count; ++t) {
    const int b = (int)(t & 1), nb2 = 1 - b;
    if (t + 1 < count) {
      if (t >= 1) CT_CUDA_TRY(cudaStreamWaitEvent(p.cs, p.freed[nb2], 0));  // block t-1 is done with it
      if ((st = load(seq[t + 1], buf[nb2], p.cs)) != CT_OK) return st;
      CT_CUDA_TRY(cudaEventRecord(p.loaded[nb2], p.cs));
    }
    CT_CUDA_TRY(cudaStreamWaitEvent(s, p.loaded[b], 0));
    if ((st = use(seq[t], buf[b])) != CT_OK) return st;
    CT_CUDA_TRY(cudaEventRecord(p.freed[b], s));
  }
  return CT_OK;
}

// Q_I^T C for the panels of block column I held in buf (rows at global
// offsets), C = rows [I*bw, m) of a device matrix whose row r is C0[r].
ct_status apply_block_column(const ct_factor* f, int64_t I, const double* buf, int64_t ldm, double* C0, int64_t ldc,
                             int64_t nc, double* work, size_t work_elems, int sms, cudaStream_t s) {
  const int64_t c0 = I * f->ooc_bw, c1 = c0 + f->ooc_bw < f->n ? c0 + f->ooc_bw : f->n;
  for (int64_t j0 = c0; j0 < c1; j0 += f->nb) {
    const int nbp = (int)(c1 - j0 < f->nb ? c1 - j0 : f->nb);
    ReflectorArgs a;
    a.V = buf + j0 + (j0 - c0) * ldm;
    a.v_f64 = true;
    a.ldv = ldm;
    a.T = f->T + (size_t)(j0 / f->nb) * f->nb * f->nb;
    a.ldt = f->nb;
    a.nbp = nbp;
    a.C = C0 + j0;
    a.c_f64 = true;
    a.ldc = ldc;
    a.mr = f->m - j0;
    a.nc = nc;
    a.fp32_math = false;
    ct_status st = apply_block_reflector(a, work, work_elems, sms, s);
    if (st != CT_OK) return st;
  }
  return CT_OK;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  ct_status alloc(size_t bytes) {
    if (getenv("CTQR_FAULT_NOMEM")) return CT_ERR_NOMEM;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? CT_ERR_NOMEM : CT_ERR_CUDA;
    }
    return CT_OK;
  }
};

}  // namespace

// B <- Q^T B for a factor held in host memory (B: m x k device FP64).
ct_status ooc_apply_qt(const ct_factor* f, double* B, int64_t ldb, int64_t k, cudaStream_t s) {
  if (k <= 0) return CT_OK;
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  const int64_t ldm = (f->m + 3) / 4 * 4, bw = f->ooc_bw, nblk = (f->n + bw - 1) / bw;
  DevBuf vb, wk;
  const size_t work_elems = reflector_work_elems(di.sms, f->nb, k);
  if ((st = vb.alloc((size_t)2 * ldm * bw * sizeof(double))) != CT_OK) return st;
  if ((st = wk.alloc(work_elems * sizeof(double))) != CT_OK) return st;
  double* buf[2] = {(double*)vb.p, (double*)vb.p + (size_t)ldm * bw};
  Pipe p;
  if ((st = p.init(s, f->ooc_overlap)) != CT_OK) return st;
  std::vector<int64_t> seq(nblk);
  for (int64_t I = 0; I < nblk; ++I) seq[I] = I;
  st = stream_blocks(
      seq.data(), nblk, buf, p, f->ooc_overlap, s,
      [&](int64_t I, double* b, cudaStream_t cs) {
        const int64_t c0 = I * bw;
        return copy_rows(f, b, ldm, c0, f->m, c0, (f->n - c0 < bw ? f->n - c0 : bw), true, cs);
      },
      [&](int64_t I, double* b) {
        return apply_block_column(f, I, b, ldm, B, ldb, k, (double*)wk.p, work_elems, di.sms, s);
      });
  // the buffers are released by this function: the compute stream's work on
  // them must be done first, and so must the copy stream's
  cudaError_t e = cudaStreamSynchronize(s);
  if (p.cs && e == cudaSuccess) e = cudaStreamSynchronize(p.cs);
  if (st == CT_OK && e != cudaSuccess) st = CT_ERR_CUDA;
  return st;
}

// B[0:n] <- R^{-1} B[0:n] for a factor held in host memory: R's block
// columns stream bottom-up; each one solves its diagonal block (Trsm_lunn)
// and updates the rows above it (Gemm_nn_mo).
ct_status ooc_trsm(const ct_factor* f, double* B, int64_t ldb, int64_t k, cudaStream_t s) {
  if (k <= 0) return CT_OK;
  const int64_t ldm = (f->n + 3) / 4 * 4, bw = f->ooc_bw, nblk = (f->n + bw - 1) / bw;
  DevBuf rb;
  ct_status st;
  if ((st = rb.alloc((size_t)2 * ldm * bw * sizeof(double))) != CT_OK) return st;
  double* buf[2] = {(double*)rb.p, (double*)rb.p + (size_t)ldm * bw};
  Pipe p;
  if ((st = p.init(s, f->ooc_overlap)) != CT_OK) return st;
  std::vector<int64_t> seq(nblk);
  for (int64_t t = 0; t < nblk; ++t) seq[t] = nblk - 1 - t;
  st = stream_blocks(
      seq.data(), nblk, buf, p, f->ooc_overlap, s,
      [&](int64_t I, double* b, cudaStream_t cs) {
        const int64_t c0 = I * bw, w = f->n - c0 < bw ? f->n - c0 : bw;
        return copy_rows(f, b, ldm, 0, c0 + w, c0, w, true, cs);
      },
      [&](int64_t I, double* b) {
        const int64_t c0 = I * bw, w = f->n - c0 < bw ? f->n - c0 : bw;
        ct_factor v;  // the diagonal block R_II as a w x w factor
        v.m = w;
        v.n = w;
        v.ld = ldm;
        v.nb = f->nb;
        v.store = CT_F64;
        v.F = b + c0;
        v.owns_F = false;
        ct_status r = launch_trsm(&v, B + c0, true, ldb, k, s);
        v.F = nullptr;
        if (r != CT_OK) return r;
        return launch_dense_update(b, true, ldm, (int)w, B + c0, ldb, B, true, ldb, c0, k, s);
      });
  cudaError_t e = cudaStreamSynchronize(s);
  if (p.cs && e == cudaSuccess) e = cudaStreamSynchronize(p.cs);
  if (st == CT_OK && e != cudaSuccess) st = CT_ERR_CUDA;
  return st;
}

}  // namespace ctqr

using namespace ctqr;

extern "C" ct_status ct_qr_factor_host(double* A, int64_t m, int64_t n, int64_t lda, const ct_ooc_opts* opts,
                                       ct_factor** out, void* stream) {
  if (!out) return CT_ERR_INVALID;
  *out = nullptr;
  if (!A || n < 1 || m < n || lda < m) return CT_ERR_INVALID;
  const int want = opts && opts->nb ? opts->nb : 64;
  if (want < 8 || want > 64) return CT_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceInfo di;
  ct_status st = device_info(&di);
  if (st != CT_OK) return st;
  // the widest panel (<= want) whose rows fit the panel kernel's shared memory
  const int nb = panel_width_that_fits(m, want, di, sizeof(double), false);
  size_t budget = opts ? opts->device_bytes : 0;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    CT_CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    budget = fr / 4;
  }
  // three m x bw FP64 buffers (A_K and the two streamed V blocks)
  const int64_t ldm = (m + 3) / 4 * 4;
  int64_t bw = (int64_t)(budget / (3 * (size_t)ldm * sizeof(double))) / nb * nb;
  const int64_t nfull = (n + nb - 1) / nb * nb;
  if (bw > nfull) bw = nfull;
  if (bw < nb) return CT_ERR_NOMEM;  // the budget holds no block column

  ct_factor* f = new ct_factor;
  f->m = m;
  f->n = n;
  f->nb = nb;
  f->prec = CT_PREC_F64;
  f->store = CT_F64;
  f->F = A;
  f->owns_F = false;
  f->ld = lda;
  f->F_host = true;
  f->ooc_bw = bw;
  f->ooc_overlap = !(opts && opts->no_overlap);
  f->device = di.device;
  if ((st = alloc_factor_aux(f, di)) != CT_OK) {
    free_factor(f);
    return st;
  }
  struct Guard {
    ct_factor* f;
    bool keep = false;
    ~Guard() {
      if (!keep) free_factor(f);
    }
  } guard{f};
  const int64_t np = npanels(f);
  CT_CUDA_TRY(cudaMemsetAsync(f->status, 0, sizeof(int), s));
  CT_CUDA_TRY(cudaMemsetAsync(f->T, 0, (size_t)np * nb * nb * sizeof(double), s));
  DevBuf ab, vb, wk, dg;
  const size_t work_elems = reflector_work_elems(di.sms, nb, bw);
  if ((st = ab.alloc((size_t)ldm * bw * sizeof(double))) != CT_OK ||
      (st = vb.alloc((size_t)2 * ldm * bw * sizeof(double))) != CT_OK ||
      (st = wk.alloc(work_elems * sizeof(double))) != CT_OK || (st = dg.alloc((size_t)n * sizeof(double))) != CT_OK)
    return st;
  double* Ak = (double*)ab.p;
  double* buf[2] = {(double*)vb.p, (double*)vb.p + (size_t)ldm * bw};
  double* diag = (double*)dg.p;
  Pipe p;
  if ((st = p.init(s, f->ooc_overlap)) != CT_OK) return st;
  cudaEvent_t ev_a = nullptr, ev_done = nullptr;
  struct Ev {
    cudaEvent_t* a;
    cudaEvent_t* b;
    ~Ev() {
      if (*a) cudaEventDestroy(*a);
      if (*b) cudaEventDestroy(*b);
    }
  } evg{&ev_a, &ev_done};
  CT_CUDA_TRY(cudaEventCreateWithFlags(&ev_a, cudaEventDisableTiming));
  CT_CUDA_TRY(cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming));
  cudaStream_t cs = f->ooc_overlap ? p.cs : s;
  const int64_t nblk = (n + bw - 1) / bw;
  std::vector<int64_t> seq;
  for (int64_t K = 0; K < nblk; ++K) {
    const int64_t c0 = K * bw, w = n - c0 < bw ? n - c0 : bw;
    // A_K -> HBM (after the previous block column went back to the host)
    if ((st = copy_rows(f, Ak, ldm, 0, m, c0, w, true, cs)) != CT_OK) return st;
    CT_CUDA_TRY(cudaEventRecord(ev_a, cs));
    CT_CUDA_TRY(cudaStreamWaitEvent(s, ev_a, 0));
    // the earlier block columns' reflectors, streamed and applied in order
    seq.resize(K);
    for (int64_t I = 0; I < K; ++I) seq[I] = I;
    st = stream_blocks(
        seq.data(), K, buf, p, f->ooc_overlap, s,
        [&](int64_t I, double* b, cudaStream_t st_) {
          const int64_t i0 = I * bw;
          return copy_rows(f, b, ldm, i0, m, i0, bw, true, st_);
        },
        [&](int64_t I, double* b) {
          return apply_block_column(f, I, b, ldm, Ak, ldm, w, (double*)wk.p, work_elems, di.sms, s);
        });
    if (st != CT_OK) return st;
    // factor the block column's rows c0..m in HBM
    ct_factor v = column_view(f, Ak, ldm, c0);
    for (int64_t j0 = c0; j0 < c0 + w; j0 += nb) {
      const int nbp = (int)(c0 + w - j0 < nb ? c0 + w - j0 : nb);
      double* Tp = f->T + (size_t)(j0 / nb) * nb * nb;
      if ((st = launch_panel(&v, j0, nbp, Tp, s)) != CT_OK) { v.F = nullptr; return st; }
      if (j0 + nbp < c0 + w) {
        ReflectorArgs a;
        a.V = Ak + j0 + (j0 - c0) * ldm;
        a.v_f64 = true;
        a.ldv = ldm;
        a.T = Tp;
        a.ldt = nb;
        a.nbp = nbp;
        a.C = Ak + j0 + (j0 + nbp - c0) * ldm;
        a.c_f64 = true;
        a.ldc = ldm;
        a.mr = m - j0;
        a.nc = c0 + w - j0 - nbp;
        a.fp32_math = false;
        if ((st = apply_block_reflector(a, (double*)wk.p, work_elems, di.sms, s)) != CT_OK) { v.F = nullptr; return st; }
      }
    }
    v.F = nullptr;
    k_block_diag<<<(unsigned)((w + 255) / 256), 256, 0, s>>>(Ak, ldm, c0, w, diag);
    CT_LAUNCH_CHECK();
    // A_K -> host (the copy stream follows the factorization of the block)
    CT_CUDA_TRY(cudaEventRecord(ev_done, s));
    CT_CUDA_TRY(cudaStreamWaitEvent(cs, ev_done, 0));
    if ((st = copy_rows(f, Ak, ldm, 0, m, c0, w, false, cs)) != CT_OK) return st;
  }
  // rank test on the collected diagonal (a 1 x n "matrix" with ld 0)
  {
    ct_factor d;
    d.m = m;
    d.n = n;
    d.ld = 0;
    d.store = CT_F64;
    d.F = diag;
    d.owns_F = false;
    d.status = f->status;
    st = launch_rank_check(&d, s);
    d.F = nullptr;
    d.status = nullptr;
    if (st != CT_OK) return st;
  }
  // the buffers are released here: both streams must be done with them
  CT_CUDA_TRY(cudaStreamSynchronize(cs));
  CT_CUDA_TRY(cudaStreamSynchronize(s));
  guard.keep = true;
  *out = f;
  return CT_OK;
}
