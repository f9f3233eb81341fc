/*
 * ctqr.h -- C ABI of the GB300 (sm_103a) library for QR-based algebraic CT
 * reconstruction (Chillaron, Quintana-Orti, Vidal, Verdu: "Computed tomography
 * medical image reconstruction on affordable equipment by using out-of-core
 * techniques", arXiv 1907.01891).
 *
 * The method models CT as the linear system A X = B (Eq. (sistema)): A is the
 * M x N system matrix, a_ij the contribution of ray i to pixel j; B holds one
 * sinogram per column; X one image per column.  It factors A = QR once
 * (Eq. (QR)) and reconstructs every slice as X = R^{-1} (Q^T B) (Eq. (qr1)),
 * applying Q^T implicitly through the Householder reflectors and solving with
 * R by backward substitution (Sec. II-C-4).
 *
 * Conventions shared by every entry point:
 *  - Matrices are column-major: element (i, j) of a matrix with leading
 *    dimension ld is at ptr[i + j*ld], ld >= rows.  Base pointers must be
 *    16-byte aligned.  All matrix pointers are DEVICE pointers owned by the
 *    caller unless stated otherwise.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call only enqueues work on that stream and returns;
 *    argument errors are returned immediately.  Errors found on the device
 *    (rank deficiency, non-finite data, a wait that timed out) are written to
 *    a device status word and reported by ct_factor_status() or by the
 *    synchronous ct_reconstruct_batch().
 *  - No entry point falls back to the CPU.
 */
#ifndef CTQR_H
#define CTQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CT_OK = 0,
  CT_ERR_INVALID = 1,     /* bad argument (size, pointer, alignment, enum)   */
  CT_ERR_NOMEM = 2,       /* device allocation failed                          */
  CT_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed              */
  CT_ERR_RANK = 4,        /* R is numerically rank deficient                   */
  CT_ERR_NONFINITE = 5,   /* NaN or Inf met in the data                        */
  CT_ERR_NOCONVERGE = 6,  /* refinement hit its iteration cap                  */
  CT_ERR_TIMEOUT = 7,     /* a bounded device-side wait gave up                */
  CT_ERR_UNSUPPORTED = 8  /* valid request this build does not implement       */
} ct_status;

/* Element type of a caller-owned matrix. */
typedef enum { CT_F64 = 0, CT_F32 = 1 } ct_dtype;

/* Arithmetic of the factorization's trailing updates (the dense contraction
 * C <- C - V T^T V^T C).  Reflector scalars and T factors are always FP64;
 * FP64-stored factors compute their panels column by column in FP64,
 * FP32-stored ones by Cholesky-QR with Householder reconstruction (the 32 x 32
 * algebra in FP64, the Gram matrix and the row solves as compensated FP32 dot
 * products of about twice FP32's precision, or FP64 when their FP32 copy does
 * not fit in shared memory; a panel with kappa_1(R1) > 3e3 falls back to the
 * column-by-column FP64 panel).  CT_PREC_F64: plain FP64 everywhere, factor stored in FP64.
 * CT_PREC_F32: factor stored in FP32, updates in FP32 (CUDA cores).
 * CT_PREC_TF32: factor stored in FP32; 128-column outer blocks of 32-column
 * panels, the outer trailing updates on the tensor cores (tcgen05) in TF32 with
 * FP32 accumulation (error-compensated by default, see ct_qr_opts).
 * CT_PREC_F16X3: as CT_PREC_TF32, but each FP32 operand of the outer updates'
 * two tensor-core products is split into two FP16 parts h + l (22 significant
 * bits; the reflectors scaled by 2^8, the trailing matrix and T^T V^T C by a
 * power of two per column) and three FP16 products h h + l h + h l are
 * accumulated in FP32: about the accuracy of the three-pass TF32 split at
 * half its tensor time and operand bytes.  A reflector entry of magnitude
 * >= 192 is reported as CT_ERR_NONFINITE.  tf32_passes must be 0. */
typedef enum { CT_PREC_F64 = 0, CT_PREC_F32 = 1, CT_PREC_TF32 = 2, CT_PREC_F16X3 = 3 } ct_prec;

/* Scanner geometry (Sec. II-A and Table (scanner) describe the paper's fan-beam
 * scanner; this struct parameterises parallel and fan beams).
 *  Image: nx*ny square pixels of side `pixel`, centred on the origin; pixel
 *    j = iy*nx + ix covers [x0 + ix*pixel, x0 + (ix+1)*pixel) x [y0 + iy*pixel,
 *    y0 + (iy+1)*pixel) with x0 = -nx*pixel/2, y0 = -ny*pixel/2 (half-open, so a
 *    ray lying on a grid line belongs to the pixels above / right of it).
 *  Rays: ray = view*n_bins + bin; view v has angle a_v = angle0 +
 *    v*angle_span/n_views; c_b = bin - (n_bins-1)/2.
 *  beam 0 (parallel): offset s = c_b*det_span/n_bins; the ray passes through
 *    s*(-sin a_v, cos a_v) with direction (cos a_v, sin a_v).
 *  beam 1 (equiangular fan): source at src_iso*(cos a_v, sin a_v), fan angle
 *    g = c_b*det_span/(n_bins-1) (g = 0 if n_bins == 1), direction
 *    (-cos(a_v+g), -sin(a_v+g)).
 *  a_ij = length of ray i inside pixel j (parameter length along the unit
 *  direction). */
typedef struct {
  int beam;          /* 0 parallel, 1 fan                                       */
  int nx, ny;        /* image size in pixels                                    */
  double pixel;      /* pixel side                                              */
  int n_views;       /* projections                                             */
  int n_bins;        /* detector bins per projection                            */
  double angle0;     /* first view angle (radians)                              */
  double angle_span; /* views are spread over [angle0, angle0 + angle_span)     */
  double src_iso;    /* fan: source-to-isocentre distance                       */
  double det_span;   /* parallel: detector width; fan: total fan angle (rad)    */
  int angle_rule;    /* 0: a_v as above; 1: a_v shifted per quarter of the      */
                     /* views as Eq. (angulos) reads: by 0, +0.5, -0.25, -0.5   */
                     /* degrees for views i = v + 1 with q n_views/4 < i <=     */
                     /* (q+1) n_views/4, q = 0..3 (the printed equation is      */
                     /* garbled; its +0.5, -0.75, -0.25 taken relative to the  */
                     /* previous quarter)                                       */
} ct_geometry;

/* Options of ct_qr_factor.  NULL selects the defaults. */
typedef struct {
  int nb;          /* panel width, 1..64 (0 = choose; CT_PREC_TF32 needs a     */
                   /* power of two <= 32)                                      */
  int in_place;    /* 1: overwrite the caller's A with the factor and borrow  */
                   /*    it (A must then have the factor's storage type and   */
                   /*    stay alive until ct_factor_destroy); 0: copy A       */
  int tf32_passes; /* CT_PREC_TF32 only: 3 (default, 0 = default) splits each  */
                   /* operand into a TF32 high part and a low remainder and   */
                   /* sums three tensor-core products (close to FP32          */
                   /* accuracy); 1 uses plain TF32 (about 3 decimal digits)   */
  int outer_nb;    /* CT_PREC_TF32 only: columns per tensor-core trailing      */
                   /* update, 256 (default, 0 = default) or 128; 256 updates  */
                   /* with two 128-column halves' reflectors at once (half    */
                   /* the passes over the trailing matrix)                    */
} ct_qr_opts;

/* Opaque factorization: reflectors V and R (in the factored matrix), tau, and
 * the per-panel T factors (Q_panel = I - V T V^T), all in device memory owned
 * by the factor until ct_factor_destroy. */
typedef struct ct_factor ct_factor;

/* Options of ct_reconstruct_batch's FP64 refinement.  NULL = defaults. */
typedef struct {
  int max_iter;    /* iteration cap, all phases together (default 200)         */
  double lambda;   /* > 0: the factored system is [A_rays; lambda*I] and the A */
                   /* passed to ct_reconstruct_batch holds only its first     */
                   /* m - n rows (the lambda*I rows are applied implicitly)   */
  double tol;      /* stop when every column has ||dx_c|| <= tol*||x_c||, or   */
                   /* (CGLS) when every column's error left after the step,    */
                   /* estimated as ||dx_c|| rho/(1-rho) from the larger of the */
                   /* last two contraction ratios rho < 1/2, is below          */
                   /* tol*||x_c|| (default 1e-12)                              */
  int method;      /* 0 auto: CGLS right after X_0 when the residual of X_0 is */
                   /*   above 1e-6 ||B|| (noisy data) or lambda > 0, else      */
                   /*   classical refinement while its updates shrink at least */
                   /*   fourfold per step, then preconditioned CGLS;           */
                   /* 1 classical only; 2 CGLS only (after the first solve)     */
} ct_refine_opts;

/* Optional report of ct_reconstruct_batch. */
typedef struct {
  int iterations;        /* refinement corrections applied after the first solve */
  double last_update;    /* max_c ||dx_c|| / ||x_c|| of the last correction      */
  double residual;       /* ||B - A X||_F / ||B||_F before the last correction   */
  double ms_total;       /* wall time of the call (host clock, synchronised)     */
  double ms_build;       /* ct_reconstruct_scan only: device time of building A  */
  double ms_factor;      /* ct_reconstruct_scan only: device time of A = QR      */
  double ms_solve;       /* ct_reconstruct_scan only: device time of the solve   */
                         /* (Q^T, R^-1 and refinement, copies excluded)          */
} ct_report;

/* Per-kernel-class launch statistics (ct_profile_kernels). */
typedef struct {
  const char* name;      /* kernel class (static storage)                        */
  uint64_t launches;     /* launches since the last ct_profile_reset             */
  uint64_t timed;        /* launches bracketed by CUDA events                    */
  double ms;             /* summed device time of the timed launches             */
  double flops;          /* summed algorithmic flops of all launches             */
  double bytes;          /* summed algorithmic DRAM bytes of all launches        */
} ct_kernel_stats;

/* One system of a batch (ct_qr_solve_batched); all pointers are device
 * pointers, column-major FP64. */
typedef struct {
  int64_t m, n;   /* rows and columns, m >= n >= 1                              */
  double* A;      /* m x n, lda >= m: overwritten by its tile QR factorization  */
  int64_t lda;
  double* B;      /* m x k, ldb >= m: rows [0, n) receive X (NULL when k == 0)  */
  int64_t ldb;
  int64_t k;      /* right-hand sides (0: factor only)                          */
} ct_batch_system;

/* Options of ct_qr_solve_batched (NULL = defaults). */
typedef struct {
  int tile;       /* tile size 32 or 64; 0 = measured choice per size class,   */
                  /* cached in $CTQR_TUNE_CACHE (else ~/.cache/ctqr_tune.json) */
  int prec;       /* CT_PREC_F64 (0, default): the persistent tile-task launch */
                  /* below; CT_PREC_TF32 or CT_PREC_F16X3: each system        */
                  /* factored by the tensor-core path of ct_qr_factor in that  */
                  /* precision (TF32 widths tuned per size class)              */
                  /* and refined to the FP64 least-squares solution by         */
                  /* ct_reconstruct_batch against its FP64 A, which is then    */
                  /* left unchanged                                            */
  int no_cache;   /* CT_PREC_F64 only.  0 (default): the task list, the tile T  */
                  /* blocks and the instantiated CUDA graph of this batch's     */
                  /* sizes stay on the device after the call, and the next call */
                  /* with the same sizes and leading dimensions (any pointers)  */
                  /* only uploads the pointers and replays the graph; one shape */
                  /* is kept per process, released by the next shape or by     */
                  /* ct_qr_solve_batched_release.  1: everything is released    */
                  /* before the call returns                                   */
} ct_batch_opts;

/* Optional report of ct_qr_solve_batched. */
typedef struct {
  int tile;       /* tile size used (0 for CT_PREC_TF32)                         */
  double ms;      /* device time of the persistent launch (CT_PREC_TF32: wall    */
                  /* time of all factorizations and refinements)                 */
  int tasks;      /* tile tasks executed (CT_PREC_TF32: 0)                       */
  int iterations; /* CT_PREC_TF32: most refinement steps any system took         */
} ct_batch_report;

/* Where the caller's B and X live for ct_reconstruct_scan. */
typedef enum { CT_DEVICE_BUFFERS = 0, CT_HOST_BUFFERS = 1 } ct_buffers;

/* Human-readable name of a status code (static storage). */
const char* ct_status_str(ct_status s);

/* Library build/version string (static storage). */
const char* ct_version(void);

/* Rows and columns of the system ct_build_system writes:
 * m = n_views*n_bins (+ nx*ny when lambda > 0), n = nx*ny.
 * Returns CT_ERR_INVALID for a malformed geometry. */
ct_status ct_system_size(const ct_geometry* geom, double lambda, int64_t* m,
                         int64_t* n);

/* Build the dense system matrix A (Eq. (sistema); a_ij = length of ray i in
 * pixel j) by Siddon-style ray traversal, written in `dtype` into the caller's
 * m x n column-major device buffer A (leading dimension lda >= m, m, n from
 * ct_system_size).  Every entry of the m x n block is written (zeros included).
 * lambda > 0 appends lambda*I below the ray rows (Tikhonov stacking [A; lambda I]).
 * Lengths are computed in FP64; CT_F32 stores them rounded. */
ct_status ct_build_system(const ct_geometry* geom, ct_dtype dtype, double lambda,
                          void* A, int64_t lda, void* stream);

/* Sinograms of k images by Joseph's projector, the paper's sinogram
 * simulator (Sec. III; Joseph 1982), for data that do not come from the
 * system matrix itself (reconstructing them with the Siddon A of
 * ct_build_system carries the model mismatch of a real scan).  For the ray of
 * unit direction (dx, dy) with |dy| >= |dx| (else the same with rows and
 * columns exchanged): at every pixel row's centre line the ray lies between
 * two pixel centres of that row; the row adds p/|dy| times their linear
 * interpolation (a pixel outside the image counts as zero).  X: n x k device
 * FP64 images (pixel iy*nx + ix, ldx >= n); B: m x k device FP64 (ldb >= m,
 * rays only: no lambda rows).  Asynchronous on `stream`. */
ct_status ct_project_joseph(const ct_geometry* geom, const double* X, int64_t ldx, int64_t k, double* B,
                            int64_t ldb, void* stream);

/* Image quality of k reconstructed slices X against reference slices R
 * (Sec. II-D), both n x k device FP64 (n = nx*ny, pixel iy*nx + ix):
 * out[3c] = MSE (Eq. MSE), out[3c+1] = PSNR in dB with the reference slice's
 * maximum as peak (Eq. psnr), out[3c+2] = SSIM (Eq. ssim), out a device array
 * of 3k doubles.  SSIM's window and constants are not given in the paper:
 * 11 x 11 Gaussian window of sigma 1.5 normalised to 1, c1 = (0.01 L)^2,
 * c2 = (0.03 L)^2, L = the reference slice's max - min, averaged over the
 * pixels whose window lies inside the image (NaN when none does).
 * Asynchronous on `stream`. */
ct_status ct_image_quality(const double* X, int64_t ldx, const double* R, int64_t ldr, int nx, int ny, int64_t k,
                           double* out, void* stream);

/* Householder QR A = QR (Eq. (QR)) of the m x n (m >= n) matrix A, blocked in
 * panels of nb columns: per panel a panel factorization (reflector generation,
 * norms; arithmetic as described for ct_prec) and its T factor (the paper's "S factor" of
 * Compute_dense_QR, Sec. II-C-3), then the trailing update of the rest
 * (Apply_left_Qt_of_dense_QR) in the arithmetic `prec` selects.
 * A has type `dtype` (CT_F64 or CT_F32), leading dimension lda.  On success
 * *out receives a new factor; A is read only (unless opts->in_place).
 * Rank deficiency (|R_ii| <= max(m,n)*eps*max|R_ii|) and non-finite input are
 * reported by ct_factor_status(). */
ct_status ct_qr_factor(const void* A, ct_dtype dtype, int64_t m, int64_t n,
                       int64_t lda, ct_prec prec, const ct_qr_opts* opts,
                       ct_factor** out, void* stream);

/* Options of ct_qr_factor_host.  NULL selects the defaults. */
typedef struct {
  size_t device_bytes; /* HBM for the streamed block columns (three m x bw FP64 */
                       /* buffers decide the block width bw); 0 = a quarter of */
                       /* the free device memory                                */
  int nb;              /* panel width 8..64 (0 = 64; narrowed to what the panel  */
                       /* kernel's shared memory holds for m rows)               */
  int no_overlap;      /* 1: copies and compute on the caller's stream one after */
                       /* the other (the paper's B-OOC); 0: a copy stream loads  */
                       /* the next block column while the current one is used   */
                       /* (O-OOC, double buffered)                               */
} ct_ooc_opts;

/* Out-of-core Householder QR (Eq. (QR)) of an m x n FP64 matrix A held in
 * HOST memory (column-major, lda >= m), for systems larger than HBM: the
 * paper's out-of-core algorithm-by-blocks (Sec. II-B, II-C) with host memory
 * in place of the disk and HBM as the block cache.  Left-looking by block
 * columns of bw columns (bw from opts->device_bytes): each block column is
 * copied to HBM, every earlier block column's reflectors are streamed in
 * (double buffered on a copy stream) and applied (Apply_left_Qt_of_dense_QR),
 * the block is factored in HBM (Compute_dense_QR per panel) and copied back.
 * A is overwritten by the factor (R on and above the diagonal, reflectors
 * below) and borrowed by it: it must stay alive and unchanged until
 * ct_factor_destroy.  tau and the panel T blocks stay in HBM.  Page-locked
 * host memory lets the copies overlap the compute (pageable memory works,
 * with staged copies).  The factor works with ct_apply_qt, ct_trsm_solve and
 * ct_reconstruct_batch (FP64 right-hand sides in HBM), each streaming the
 * factor through HBM again (Q^T block columns in factorization order, R's
 * block columns bottom-up); the FP32 entry points, ct_factor_copy,
 * ct_factor_save and ct_apply_qt_noalloc return CT_ERR_UNSUPPORTED for it.
 * Synchronous on `stream`.  CT_ERR_NOMEM when device_bytes holds no block
 * column; rank and non-finite data are reported by ct_factor_status(). */
ct_status ct_qr_factor_host(double* A, int64_t m, int64_t n, int64_t lda, const ct_ooc_opts* opts,
                            ct_factor** out, void* stream);

/* Shape and arithmetic of a factor (any pointer may be NULL). */
ct_status ct_factor_info(const ct_factor* f, int64_t* m, int64_t* n, int* nb,
                         ct_prec* prec);

/* Device pointers of the factored matrix (R on and above the diagonal, the
 * reflectors below it, element type *dtype, leading dimension *ld) and of tau
 * (FP64, n entries).  The memory stays owned by the factor. */
ct_status ct_factor_data(const ct_factor* f, const void** F, ct_dtype* dtype,
                         int64_t* ld, const double** tau);

/* Copy the factored matrix (R on and above the diagonal, the reflectors' v
 * below it, v_0 = 1 implicit) into the caller's m x n device buffer F_out
 * (element type = the factor's storage type from ct_factor_data, leading
 * dimension ld_out >= m) and tau into the caller's n-element FP64 device
 * buffer tau_out (either output may be NULL).  Asynchronous on `stream`. */
ct_status ct_factor_copy(const ct_factor* f, void* F_out, int64_t ld_out, double* tau_out,
                         void* stream);

/* Synchronise `stream` and return the device status recorded by the work of
 * this factor so far (CT_OK, CT_ERR_RANK, CT_ERR_NONFINITE, CT_ERR_TIMEOUT). */
ct_status ct_factor_status(const ct_factor* f, void* stream);

/* B <- Q^T B in place for the m x k FP64 device matrix B (ldb >= m): the first
 * sub-step of X = R^{-1}(Q^T B) (Eq. (qr1)), applying each panel's block
 * reflector I - V T^T V^T in factorization order (the Apply_left_Qt tasks of
 * the solve, Sec. II-C-4).  k may be 0 (no-op). */
ct_status ct_apply_qt(const ct_factor* f, double* B, int64_t ldb, int64_t k,
                      void* stream);

/* B <- Q^T B in place in FP32 arithmetic for the m x k FP32 device matrix B
 * (ldb >= m, B 16-byte aligned) with a CT_PREC_F32 / CT_PREC_TF32 factor: the
 * first sub-step of Eq. (qr1) at the factor's precision, as the refinement's
 * first solve X_0 uses it.  Two-level (TF32) factors with 1 <= k <= 32 apply
 * all their 128-column outer blocks in one cooperative launch when each SM's
 * share of the rows fits its shared memory (about 160 rows per SM), else
 * block by block.  CT_ERR_UNSUPPORTED for an FP64 factor; k may be 0. */
ct_status ct_apply_qt_f32(const ct_factor* f, float* B, int64_t ldb, int64_t k,
                          void* stream);

/* B <- Q^T B exactly like ct_apply_qt, for callers that cannot let a library
 * allocate device memory: applications whose framework has already reserved
 * the GPU's memory for its own caching allocator (an allocation here would
 * fail), or latency-critical loops that cannot afford the synchronisation an
 * allocation implies.  The paper has no counterpart; this is a deployment
 * variant of the Q^T step.
 * Its workspace is a fixed 2.03 MiB array in the library's static device
 * memory, held by every GPU that loads the library until the process exits;
 * it calls no allocation routine.  Limit: k <= 64 right-hand sides per call;
 * a larger k returns CT_ERR_INVALID (split B into column blocks).  The first
 * call on each device looks up the array's device address and caches it;
 * make that first call before any stream capture.  The cached address
 * belongs to the device's primary context: after cudaDeviceReset it is stale,
 * so do not use this entry point on a device that was reset.  All calls share the one
 * array and it keeps the last call's contents (nothing in it needs clearing:
 * each call writes what it reads), so calls that overlap on the GPU -- on
 * different streams, threads or factors -- race and corrupt each other's
 * results: serialise them.  Launch timing (ct_profile_enable) must stay off:
 * it creates CUDA events. */
ct_status ct_apply_qt_noalloc(const ct_factor* f, double* B, int64_t ldb, int64_t k, void* stream);

/* B[0:n, 0:k] <- R^{-1} B[0:n, 0:k] in place (FP64): backward substitution
 * with the factor's upper triangular R, by blocks: a triangular solve of each
 * diagonal block (Trsm_lunn) followed by the update of the blocks above it
 * (Gemm_nn_mo), Sec. II-C-4.  ldb >= n. */
ct_status ct_trsm_solve(const ct_factor* f, double* B, int64_t ldb, int64_t k,
                        void* stream);

/* The preconditioner solves of the mixed-precision refinement, exposed on
 * their own: B[0:n, 0:k] <- R^{-1} B (transpose = 0) or R^{-T} B
 * (transpose != 0) in FP32 arithmetic with the FP32-stored R of a
 * CT_PREC_F32 / CT_PREC_TF32 factor; B is an FP32 device matrix, ldb >= n.
 * The paper's factor is FP64 and has no counterpart; the operation is the
 * back substitution of Sec. II-C-4 at lower precision.  For k <= 64 one
 * persistent launch walks the 128-row block rows in dependency order (each
 * block of R read once for all k columns), each block row finished by a
 * product with its inverted diagonal block; wider B uses recursive halving
 * with one product per split.
 * CT_ERR_UNSUPPORTED for an FP64 factor. */
ct_status ct_trsm_solve_f32(const ct_factor* f, float* B, int64_t ldb, int64_t k, int transpose,
                            void* stream);

/* X = R^{-1} (Q^T B)[0:n] for k slices (Eq. (qr1)): B is m x k (ldb >= m,
 * read only), X is n x k (ldx >= n), both FP64 device matrices.
 * Without A (A == NULL) this is one Q^T application and one back-solve in
 * FP64 arithmetic with the factor as stored.
 * With A (the original m x n system matrix, type A_dtype, leading dimension
 * lda; FP64 for full accuracy) the result is refined with FP64 residuals
 * until every column satisfies ||dx_c|| <= tol ||x_c||.  This is how a
 * CT_PREC_F32 / CT_PREC_TF32 factor reaches FP64 accuracy.
 *  - classical refinement: X_0 = R^{-1}(Q^T B)[0:n]; repeat Res = B - A X
 *    (FP64), D = R^{-1}(Q^T Res)[0:n] (FP32 arithmetic for an FP32-stored
 *    factor, FP64 otherwise), X += D.  Cheap; exact for consistent B
 *    (B = A X), but for noisy B the rounding of the correction solve, which is
 *    proportional to the residual, stops it short of the least-squares
 *    solution.
 *  - CGLS on min ||A R^{-1} y - B||, X = R^{-1} y (the low-precision R as a
 *    right preconditioner), every product with A, A^T, R^{-1}, R^{-T} in FP64:
 *    converges to the least-squares solution for any B.
 * Synchronous: returns once X holds the result, with the factor's device
 * status, or CT_ERR_NOCONVERGE if the cap was reached (X then holds the last
 * iterate).  `report` (may be NULL) receives iteration counts and timings. */
ct_status ct_reconstruct_batch(const ct_factor* f, const void* A,
                               ct_dtype A_dtype, int64_t lda, const double* B,
                               int64_t ldb, double* X, int64_t ldx, int64_t k,
                               const ct_refine_opts* ropts, ct_report* report,
                               void* stream);

/* Tensor-core contraction used by the trailing update (the paper's
 * Apply_left_Qt_of_dense_QR task, Sec. II-C-3, applies a block reflector
 * C - V T^T V^T C through two such products): C = A^T B (accumulate == 0) or
 * C -= A^T B (accumulate == 1), with A K x M, B K x N and C M x N, all FP32
 * column-major device matrices (lda >= K and ldb >= K multiples of 4, A and B
 * 16-byte aligned, ldc >= M).  tcgen05 TF32 MMAs with FP32 accumulation;
 * split3 = 1 splits each operand into a TF32 high part and a low remainder
 * and sums hi*hi + hi*lo + lo*hi, recovering close to FP32 accuracy at three
 * times the tensor work.  Asynchronous on `stream`; a timed-out device wait
 * is reported as CT_ERR_TIMEOUT by the next ct_gemm_status call. */
ct_status ct_gemm_tf32_tn(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                          const float* B, int64_t ldb, float* C, int64_t ldc, int accumulate,
                          int split3, void* stream);

/* The same contraction with each FP32 operand split into two FP16 parts (the
 * products of CT_PREC_F16X3 factors): A scaled by 2^8 (|A| < 128 required),
 * B per column by a power of two from its largest magnitude; C = A^T B
 * (accumulate == 0: the split-K product kernel, B split on chip) or C -= A^T B
 * (accumulate == 1: the persistent update kernel, both operands split first;
 * K <= 256).  M, N <= 65535; lda, ldb multiples of 4, A and B 16-byte
 * aligned.  Allocates its split operands on `stream`.  Errors as
 * ct_gemm_tf32_tn (CT_ERR_NONFINITE is not checked here). */
ct_status ct_gemm_f16x3_tn(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda,
                           const float* B, int64_t ldb, float* C, int64_t ldc, int accumulate,
                           void* stream);

/* Synchronise `stream` and return (and clear) the device status recorded by
 * ct_gemm_tf32_tn and ct_gemm_f16x3_tn calls. */
ct_status ct_gemm_status(void* stream);

/* Whole method for one scan: build A from `geom` on the device (Eq.
 * (sistema), stacked over lambda*I when lambda > 0), factor it (Eq. (QR)) with
 * trailing updates in `prec`, and reconstruct the k slices X = R^{-1}(Q^T B)
 * (Eq. (qr1)), refined with FP64 residuals against the FP64 A when prec is not
 * CT_PREC_F64.  B is m x k FP64 (ldb >= m), X is n x k FP64 (ldx >= n), both in
 * host memory (CT_HOST_BUFFERS: copied in and out inside the call; page-locked
 * memory gives full copy bandwidth) or in device memory (CT_DEVICE_BUFFERS).
 * All other device memory (A in FP64, the factor, scratch) is allocated and
 * released inside the call.  Synchronous; `report` (may be NULL) receives the
 * phase timings. */
ct_status ct_reconstruct_scan(const ct_geometry* geom, double lambda, ct_prec prec,
                              const double* B, int64_t ldb, double* X, int64_t ldx,
                              int64_t k, ct_buffers where, const ct_refine_opts* ropts,
                              ct_report* report, void* stream);

/* Launch accounting.  Every kernel launch is counted; with timing enabled
 * each launch is also bracketed by CUDA events on its stream. */
void ct_profile_enable(int on);
/* Zero the counters (synchronises pending timing events first). */
void ct_profile_reset(void);
/* Fill up to max_entries stats (one per kernel class) and return how many
 * were written; out == NULL returns the number of classes.  Synchronises the
 * pending timing events. */
int ct_profile_kernels(ct_kernel_stats* out, int max_entries);
/* Total kernel launches since the last reset. */
uint64_t ct_kernel_launches(void);

/* Factor and solve `count` independent least-squares systems of any sizes
 * in one persistent launch: each A_s = Q_s R_s by the paper's algorithm-by-
 * blocks (Sec. II-C-3: Compute_dense_QR, Apply_left_Qt_of_dense_QR,
 * Compute_TD_QR and Apply_left_Qt_of_TD_QR on b x b tiles, Table
 * tasks_qr_ab), then X_s = R_s^{-1}(Q_s^T B_s) by the solve tasks of Table
 * tasks_solve_ab (the two Apply tasks on B, Trsm_lunn, Gemm_nn_mo).  The tasks
 * of all systems share one device work queue consumed by one CTA per SM, with
 * per-tile version counters ordering them (bounded waits); the task list is
 * built on the host and uploaded once per batch shape, and the upload of the
 * systems' pointers, the counter resets and the launch form one CUDA graph,
 * instantiated once per shape and replayed by later calls of that shape (see
 * ct_batch_opts.no_cache).  FP64 throughout.  `systems` is a host
 * array; A_s and B_s are overwritten.  Synchronous: returns when done, with
 * CT_ERR_RANK / CT_ERR_NONFINITE / CT_ERR_TIMEOUT if any system hit one.
 * Stack lambda*I under a rank-deficient A with ct_build_system. */
ct_status ct_qr_solve_batched(int count, const ct_batch_system* systems, const ct_batch_opts* opts,
                              ct_batch_report* report, void* stream);
/* Free the device memory (task list, tile T blocks, counters) and the CUDA
 * graph that ct_qr_solve_batched keeps for the last batch shape; the next call
 * plans again.  Safe to call at any time, also when nothing is kept. */
void ct_qr_solve_batched_release(void);
/* The tile-task list ct_qr_solve_batched executes for these systems with tile
 * size `tile` (32 or 64), built on the host only (no device work; the
 * systems' A and B pointers are not read and may be NULL).  The tasks are the
 * GEQRT / UNMQR / TSQRT / TSMQR tasks of Table tasks_qr_ab and the solve
 * tasks of Table tasks_solve_ab in the order the persistent launch takes
 * them.  Each task is 25 int32 in `tasks` (caller-owned, room for max_tasks
 * records; NULL: only the counts): type (0 GEQRT, 1 UNMQR, 2 TSQRT, 3 TSMQR,
 * 4 UNMQR on B, 5 TSMQR on B, 6 Trsm_lunn, 7 Gemm_nn_mo), system, i, j, k,
 * the number of dependencies nd and of increments ni, then six dependency
 * counters (-1 past nd), the six versions they must reach before the task
 * runs, and six counters the task increments when done (-1 past ni).  Counter
 * 2p counts the writes of tile part p, counter 2p + 1 its reads; *ntasks and
 * *nparts (may be NULL) receive the task and part counts.  CT_ERR_INVALID
 * for malformed systems or too small a buffer, CT_ERR_UNSUPPORTED beyond
 * 2^31 - 1 tasks. */
ct_status ct_batch_plan(int count, const ct_batch_system* systems, int tile, int32_t* tasks, int64_t max_tasks,
                        int64_t* ntasks, int* nparts);

/* A factor kept beyond the process.  The paper computes the factorization
 * once and stores it so that every later batch of slices reuses it (Sec.
 * II-B; its factor is kept on disk as tile files).  ct_factor_save writes the
 * factored matrix, tau, the panel T blocks and (CT_PREC_TF32) the per-block
 * V^T V and T stores to one file: a 128-byte header (magic "CTQRFAC1",
 * version, m, n, nb, prec, storage type, `tag`, payload size, FNV-1a-64
 * checksum of the payload) followed by the arrays, column-major with
 * leading dimension m.  `tag` is the caller's identifier of what was
 * factored (e.g. ct_geometry_hash of the scan), 0 for none.  The copies go
 * through a 64 MiB page-locked host buffer in chunks; synchronous on
 * `stream`.  Errors: CT_ERR_INVALID for a NULL argument or a file that
 * cannot be written; CT_ERR_CUDA / CT_ERR_NOMEM from the copies. */
ct_status ct_factor_save(const ct_factor* f, const char* path, uint64_t tag, void* stream);

/* Read a file written by ct_factor_save into a new factor on the current
 * device (*out; release with ct_factor_destroy).  *tag (may be NULL)
 * receives the stored tag.  Synchronous on `stream`.  CT_ERR_INVALID when
 * the file is missing, its header is malformed or inconsistent, its size is
 * not the header's, or the payload checksum does not match (nothing is
 * returned then); CT_ERR_NOMEM when the factor does not fit. */
ct_status ct_factor_load(const char* path, ct_factor** out, uint64_t* tag, void* stream);

/* Shape, arithmetic and tag of a factor file, from its header alone (no GPU
 * needed; any output may be NULL).  CT_ERR_INVALID as for ct_factor_load's
 * header checks. */
ct_status ct_factor_file_info(const char* path, int64_t* m, int64_t* n, int* nb, ct_prec* prec,
                              uint64_t* tag);

/* A 64-bit FNV-1a hash of a geometry and its lambda (every field, +0 and -0
 * alike), never 0: a tag that ties a saved factor to the scan it factors.
 * Returns 0 for NULL. */
uint64_t ct_geometry_hash(const ct_geometry* geom, double lambda);

/* Release a factor and its device memory (NULL is a no-op).  Waits for the
 * device to finish all queued work first, so a factor may be destroyed while
 * kernels that use it are still in flight. */
void ct_factor_destroy(ct_factor* f);

/* ------------------------------------------------------------------------
 * Learned surrogate.  The paper has no learned part: it reconstructs every
 * slice as the least-squares solution X = R^{-1} (Q^T B)[0:n] of Eq. (qr1) with
 * the factor of Eq. (QR).  These entry points add a small convolutional
 * network that maps the backprojection g = A^T b of one sinogram (A built as
 * in Sec. II-A) to an image estimate x_hat, and a gate that accepts x_hat only
 * when its FP64 data residual ||A x_hat - b|| / ||b|| is at most a tolerance;
 * every slice that fails is solved through a QR factor instead, so the output
 * is the QR solution wherever the network is not good enough.
 *
 * Network (images nx x ny, pixel j = iy * nx + ix as in the columns of A;
 * 3x3 kernels, stride 1, zero padding 1; C = 32 channels, 6 layers):
 *   a1 = relu(conv1(in_scale * g))             1 -> C
 *   a_l = a_{l-1} + relu(conv_l(a_{l-1}))      l = 2..5, C -> C
 *   x_hat = out_scale * conv6(a5)              C -> 1
 * Weights and activations are stored in BF16, products accumulate in FP32.
 * Parameters are one FP32 vector; layer l holds its weights [out][in][3][3]
 * followed by its out biases, layers in order (ct_surrogate_num_params
 * gives the length).  Training minimises the mean over pixels and images of
 * (y - x / out_scale)^2, y the network output, with Adam (beta1 0.9, beta2
 * 0.999, eps 1e-8) on the FP32 parameters; the BF16 copy is refreshed after
 * each step.  All images are FP64, column-major n x k with ld = n.
 * Errors: CT_ERR_INVALID for bad sizes or NULL pointers; CT_ERR_NOMEM when an
 * activation buffer cannot be allocated; CT_ERR_CUDA otherwise.
 * ------------------------------------------------------------------------ */
typedef struct ct_surrogate ct_surrogate;

typedef struct {
  double in_scale;   /* network input = in_scale * A^T b                     */
  double out_scale;  /* x_hat = out_scale * network output                  */
  uint64_t seed;     /* seeds the uniform initialisation of the weights     */
} ct_surrogate_opts;

typedef struct {
  int64_t slices;        /* k                                                 */
  int64_t fallbacks;     /* slices that failed the gate                       */
  double max_residual;   /* largest gate residual among the accepted slices   */
  double ms_total;       /* host wall time of the call                        */
  double ms_network;     /* device time: backprojection + network             */
  double ms_gate;        /* device time: FP64 residuals and compaction        */
  double ms_fallback;    /* device time: QR solve of the failing slices       */
} ct_surrogate_report;

/* Create a network for the geometry g (fan or parallel beam, Sec. II-A); the
 * exact FP64 sparse A of g is built once and kept for backprojections and
 * gates.  *out receives the handle (free with ct_surrogate_destroy). */
ct_status ct_surrogate_init(const ct_geometry* g, const ct_surrogate_opts* opts, ct_surrogate** out);
int64_t ct_surrogate_num_params(const ct_surrogate* s);
/* Copy the FP32 parameters to host (set = 0) or from host (set != 0). */
ct_status ct_surrogate_params(ct_surrogate* s, float* host, int set);
/* G = A^T B for k sinograms B (device FP64, m rays x k, ldb >= m); G is
 * device FP64 n x k with ld = n. */
ct_status ct_surrogate_backproject(ct_surrogate* s, const double* B, int64_t ldb, int64_t k, double* G,
                                   void* stream);
/* B = A X for k images X (device FP64 n x k, ld = n): the sinograms of
 * Eq. (sistema) computed with the exact sparse A; B device FP64, ldb >= m. */
ct_status ct_surrogate_project(ct_surrogate* s, const double* X, int64_t k, double* B, int64_t ldb,
                               void* stream);
/* One Adam step on a batch: inputs G (backprojections) and targets X, both
 * device FP64 n x batch.  *loss (may be NULL) receives the batch loss before
 * the step. */
ct_status ct_surrogate_train_step(ct_surrogate* s, const double* G, const double* X, int64_t batch, float lr,
                                  double* loss, void* stream);
/* Loss and gradient (host FP32, ct_surrogate_num_params entries, may be
 * NULL) of a batch, without changing the parameters. */
ct_status ct_surrogate_grad(ct_surrogate* s, const double* G, const double* X, int64_t batch, double* loss,
                            float* grad_host, void* stream);
/* x_hat for backprojections G (device FP64 n x k): the network alone. */
ct_status ct_surrogate_forward(ct_surrogate* s, const double* G, double* Xhat, int64_t k, void* stream);
/* Gated reconstruction of k sinograms B (device FP64, ldb >= m rays): X
 * (device FP64, ldx >= n) receives x_hat for the slices whose FP64 residual
 * ||A x_hat - b|| / ||b|| <= tol (||A x_hat|| when b = 0), and for the others
 * the solution through the factor f of A (or of [A; lambda I] with
 * ropts->lambda > 0; refined when f is a mixed-precision factor, as
 * ct_reconstruct_scan does).  f may be NULL: failing slices then keep x_hat.
 * resid (device, k doubles, may be NULL) receives every slice's gate
 * residual (NaN or Inf fail the gate).  Returns the fallback solve's status
 * when it fails. */
ct_status ct_surrogate_infer(ct_surrogate* s, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t k,
                             double tol, const ct_factor* f, const ct_refine_opts* ropts, double* resid,
                             ct_surrogate_report* report, void* stream);
void ct_surrogate_destroy(ct_surrogate* s);

#ifdef __cplusplus
}
#endif

#endif /* CTQR_H */
