// sparse.cu -- exact FP64 products with the system matrix for the refinement.
//
// A CT system matrix is very sparse: ray i crosses at most nx + ny of the
// nx*ny pixels (Eq. (sistema), a_ij = length of ray i in pixel j).  The
// refinement needs r = b - A x and A^T r in FP64 at every iteration; with the
// dense A those are 2mnk flops each, at the FP64 rate of this GPU the most
// expensive part of the whole method.  Here A is kept in compressed form,
// built by the same ray traversal that writes the dense matrix (the entries
// are bitwise the same), and applied with row-major sparse x dense products:
//   CSR (ray -> pixels)   for A X,     CSC (pixel -> rays)  for A^T R.
// The CSC is produced by a counting scatter followed by a sort of every column
// by ray index, so its entry order -- and every sum -- is deterministic.
#include "internal.cuh"

namespace ctqr {

ct_status launch_ray_nnz(const ct_geometry* gg, int* nnz, cudaStream_t s);
ct_status launch_ray_fill(const ct_geometry* gg, const int64_t* row_ptr, int* col, double* val, cudaStream_t s);

namespace {

// Exclusive prefix sum of L ints into L+1 int64 (single CTA, 1024 threads).
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ in, int64_t L, int64_t* __restrict__ out) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t per = (L + 1023) / 1024;
  const int64_t b = t * per, e = b + per < L ? b + per : L;
  int64_t s = 0;
  for (int64_t i = b; i < e; ++i) s += in[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int64_t v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int64_t run = part[t] - s;  // exclusive prefix of this chunk
  for (int64_t i = b; i < e; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (t == 1023) out[L] = part[1023];
}

__global__ void k_count_cols(const int64_t* __restrict__ row_ptr, const int* __restrict__ col, int64_t rows,
                             int* __restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) atomicAdd(&cnt[col[e]], 1);
}

__global__ void k_scatter_cols(const int64_t* __restrict__ row_ptr, const int* __restrict__ col,
                               const double* __restrict__ val, int64_t rows, int* __restrict__ cursor,
                               int* __restrict__ crow, double* __restrict__ cval) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x)
    for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
      const int pos = atomicAdd(&cursor[col[e]], 1);
      crow[pos] = (int)i;
      cval[pos] = val[e];
    }
}

__global__ void k_int64_to_int(const int64_t* __restrict__ in, int64_t L, int* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) out[i] = (int)in[i];
}

// Sort every column segment by ray index (bitonic sort in shared memory,
// segments up to kMaxSeg entries; longer ones are reported).
constexpr int kMaxSeg = 4096;
__global__ void __launch_bounds__(256) k_sort_cols(const int64_t* __restrict__ col_ptr, int* __restrict__ crow,
                                                   double* __restrict__ cval, int* status) {
  __shared__ int key[kMaxSeg];
  __shared__ double v[kMaxSeg];
  const int64_t b = col_ptr[blockIdx.x], e = col_ptr[blockIdx.x + 1];
  const int len = (int)(e - b);
  if (len <= 1) return;
  if (len > kMaxSeg) {
    if (threadIdx.x == 0) set_status(status, CT_ERR_UNSUPPORTED);
    return;
  }
  int p2 = 1;
  while (p2 < len) p2 <<= 1;
  for (int i = threadIdx.x; i < p2; i += blockDim.x) {
    key[i] = i < len ? crow[b + i] : 0x7fffffff;
    v[i] = i < len ? cval[b + i] : 0.0;
  }
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          if ((key[i] > key[l]) == up) {
            const int tk = key[i]; key[i] = key[l]; key[l] = tk;
            const double tv = v[i]; v[i] = v[l]; v[l] = tv;
          }
        }
      }
      __syncthreads();
    }
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    crow[b + i] = key[i];
    cval[b + i] = v[i];
  }
}

// Yr[i, :] = sum_e val[e] * Xr[idx[e], :] for row-major Xr (ld k) and Yr;
// one warp per output row, lanes across the k right-hand sides.
__global__ void __launch_bounds__(256) k_spmm(const int64_t* __restrict__ ptr, const int* __restrict__ idx,
                                              const double* __restrict__ val, int64_t rows,
                                              const double* __restrict__ Xr, int k, double* __restrict__ Yr) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < rows; i += nwarps) {
    const int64_t b = ptr[i], e = ptr[i + 1];
    for (int c0 = 0; c0 < k; c0 += 64) {
      const int ca = c0 + lane, cb = c0 + 32 + lane;
      double acc0 = 0.0, acc1 = 0.0;
      for (int64_t q = b; q < e; ++q) {
        const int j = __ldg(idx + q);
        const double a = __ldg(val + q);
        const double* xr = Xr + (int64_t)j * k;
        if (ca < k) acc0 += a * xr[ca];
        if (cb < k) acc1 += a * xr[cb];
      }
      if (ca < k) Yr[i * k + ca] = acc0;
      if (cb < k) Yr[i * k + cb] = acc1;
    }
  }
}

// The same product for k <= 16: the two half-warps take the even and the odd
// nonzeros of the row (lane c = lane % 16 the column) and are added at the
// end, so every lane of the FP64 pipe's warp instructions does work (on GB300
// an FP64 warp instruction costs its full issue time whatever its mask).
__global__ void __launch_bounds__(256) k_spmm16(const int64_t* __restrict__ ptr, const int* __restrict__ idx,
                                                const double* __restrict__ val, int64_t rows,
                                                const double* __restrict__ Xr, int k, double* __restrict__ Yr) {
  const int lane = threadIdx.x & 31, h = lane >> 4, c = lane & 15;
  const bool act = c < k;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < rows; i += nwarps) {
    const int64_t b = ptr[i], e = ptr[i + 1];
    double acc = 0.0;
    int64_t q = b + h;
    for (; q + 6 < e; q += 8) {  // four nonzeros per half-warp in flight
      int j[4];
      double a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        j[u] = __ldg(idx + q + 2 * u);
        a[u] = __ldg(val + q + 2 * u);
      }
      double x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = act ? Xr[(int64_t)j[u] * k + c] : 0.0;
#pragma unroll
      for (int u = 0; u < 4; ++u) acc += a[u] * x[u];
    }
    for (; q < e; q += 2) {
      const int j = __ldg(idx + q);
      const double a = __ldg(val + q);
      if (act) acc += a * Xr[(int64_t)j * k + c];
    }
    acc += __shfl_down_sync(0xffffffffu, acc, 16);
    if (h == 0 && act) Yr[i * k + c] = acc;
  }
}

// Column-major <-> row-major for rows x k FP64 blocks through 32 x 32 tiles.
// mode 0: dst = src, 1: dst -= src, 2: dst = -src (row-major -> column-major only).
__global__ void __launch_bounds__(256) k_to_rows(const double* __restrict__ src, int64_t ld, int64_t rows, int k,
                                                 double* __restrict__ dst) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int rr = e % 32, cc = e / 32;
    if (r0 + rr < rows && c0 + cc < k) t[rr][cc] = src[r0 + rr + (int64_t)(c0 + cc) * ld];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int cc = e % 32, rr = e / 32;
    if (r0 + rr < rows && c0 + cc < k) dst[(r0 + rr) * k + c0 + cc] = t[rr][cc];
  }
}

__global__ void __launch_bounds__(256) k_from_rows(const double* __restrict__ src, int64_t rows, int k,
                                                   double* __restrict__ dst, int64_t ld, int mode) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int cc = e % 32, rr = e / 32;
    if (r0 + rr < rows && c0 + cc < k) t[rr][cc] = src[(r0 + rr) * k + c0 + cc];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 1024; e += 256) {
    const int rr = e % 32, cc = e / 32;
    if (r0 + rr < rows && c0 + cc < k) {
      double* d = dst + r0 + rr + (int64_t)(c0 + cc) * ld;
      if (mode == 0) *d = t[rr][cc];
      else if (mode == 1) *d -= t[rr][cc];
      else *d = -t[rr][cc];
    }
  }
}

}  // namespace

SparseSystem::~SparseSystem() { release(); }

void SparseSystem::release() {
  for (void* p : {(void*)row_ptr, (void*)col, (void*)val, (void*)col_ptr, (void*)crow, (void*)cval, (void*)stage})
    if (p) cudaFree(p);
  row_ptr = col_ptr = nullptr;
  col = crow = nullptr;
  val = cval = stage = nullptr;
}

ct_status SparseSystem::build(const ct_geometry* g, int64_t k_max, int* status, cudaStream_t s) {
  release();
  m = (int64_t)g->n_views * g->n_bins;
  n = (int64_t)g->nx * g->ny;
  kmax = k_max;
  int* cnt = nullptr;
  const size_t cnt_elems = (size_t)(m > n ? m : n) + 1;
  CT_CUDA_TRY(cudaMalloc(&cnt, cnt_elems * sizeof(int)));
  struct Free { int* p; ~Free() { cudaFree(p); } } fr{cnt};
  CT_CUDA_TRY(cudaMalloc(&row_ptr, (size_t)(m + 1) * sizeof(int64_t)));
  ct_status st;
  if ((st = launch_ray_nnz(g, cnt, s)) != CT_OK) return st;
  {
    LaunchScope ls(K_COPY, s, 0.0, 12.0 * m);
    k_scan<<<1, 1024, 0, s>>>(cnt, m, row_ptr);
    CT_LAUNCH_CHECK();
  }
  CT_CUDA_TRY(cudaMemcpyAsync(&nnz, row_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  CT_CUDA_TRY(cudaStreamSynchronize(s));
  const size_t nz = (size_t)(nnz > 0 ? nnz : 1);
  CT_CUDA_TRY(cudaMalloc(&col, nz * sizeof(int)));
  CT_CUDA_TRY(cudaMalloc(&val, nz * sizeof(double)));
  if ((st = launch_ray_fill(g, row_ptr, col, val, s)) != CT_OK) return st;
  // CSC
  CT_CUDA_TRY(cudaMalloc(&col_ptr, (size_t)(n + 1) * sizeof(int64_t)));
  CT_CUDA_TRY(cudaMalloc(&crow, nz * sizeof(int)));
  CT_CUDA_TRY(cudaMalloc(&cval, nz * sizeof(double)));
  CT_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)n * sizeof(int), s));
  {
    LaunchScope ls(K_COPY, s, 0.0, 8.0 * nnz);
    k_count_cols<<<512, 256, 0, s>>>(row_ptr, col, m, cnt);
    CT_LAUNCH_CHECK();
    k_scan<<<1, 1024, 0, s>>>(cnt, n, col_ptr);
    CT_LAUNCH_CHECK();
  }
  // cursor[j] starts at col_ptr[j] (int: nnz < 2^31 is checked)
  if (nnz >= (int64_t)INT32_MAX) return CT_ERR_UNSUPPORTED;
  int* cursor = cnt;
  {
    LaunchScope ls(K_COPY, s, 0.0, 12.0 * n);
    k_int64_to_int<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(col_ptr, n, cursor);
    CT_LAUNCH_CHECK();
  }
  {
    LaunchScope ls(K_COPY, s, 0.0, 36.0 * nnz);
    k_scatter_cols<<<512, 256, 0, s>>>(row_ptr, col, val, m, cursor, crow, cval);
    CT_LAUNCH_CHECK();
    k_sort_cols<<<(unsigned)n, 256, 0, s>>>(col_ptr, crow, cval, status);
    CT_LAUNCH_CHECK();
  }
  CT_CUDA_TRY(cudaMalloc(&stage, (size_t)2 * (m > n ? m : n) * (k_max > 0 ? k_max : 1) * sizeof(double)));
  return CT_OK;
}

// Y[0:m, 0:k] (column-major, ldy) op= A X with X n x k column-major (ldx):
// mode 0 store, 1 subtract, 2 store negated.
ct_status SparseSystem::apply(const double* X, int64_t ldx, int64_t k, double* Y, int64_t ldy, int mode,
                              cudaStream_t s) const {
  if (k <= 0) return CT_OK;
  if (k > kmax) return CT_ERR_INVALID;
  double* Xr = stage;
  double* Yr = stage + (size_t)(m > n ? m : n) * kmax;
  const dim3 tb(256);
  {
    LaunchScope ls(K_COPY, s, 0.0, 16.0 * n * k);
    k_to_rows<<<dim3((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32)), tb, 0, s>>>(X, ldx, n, (int)k, Xr);
    CT_LAUNCH_CHECK();
  }
  {
    LaunchScope ls(K_SPMM, s, 2.0 * nnz * k, 12.0 * nnz + 8.0 * (m + n) * k);
    const unsigned g = (unsigned)((m + 7) / 8 < 65535 ? (m + 7) / 8 : 65535);
    if (k <= 16) k_spmm16<<<g, tb, 0, s>>>(row_ptr, col, val, m, Xr, (int)k, Yr);
    else k_spmm<<<g, tb, 0, s>>>(row_ptr, col, val, m, Xr, (int)k, Yr);
    CT_LAUNCH_CHECK();
  }
  {
    LaunchScope ls(K_COPY, s, 0.0, 16.0 * m * k);
    k_from_rows<<<dim3((unsigned)((m + 31) / 32), (unsigned)((k + 31) / 32)), tb, 0, s>>>(Yr, m, (int)k, Y, ldy, mode);
    CT_LAUNCH_CHECK();
  }
  return CT_OK;
}

// S[0:n, 0:k] = A^T R with R m x k column-major (ldr), S column-major (lds).
ct_status SparseSystem::apply_t(const double* R, int64_t ldr, int64_t k, double* S, int64_t lds,
                                cudaStream_t s) const {
  if (k <= 0) return CT_OK;
  if (k > kmax) return CT_ERR_INVALID;
  double* Rr = stage;
  double* Sr = stage + (size_t)(m > n ? m : n) * kmax;
  const dim3 tb(256);
  {
    LaunchScope ls(K_COPY, s, 0.0, 16.0 * m * k);
    k_to_rows<<<dim3((unsigned)((m + 31) / 32), (unsigned)((k + 31) / 32)), tb, 0, s>>>(R, ldr, m, (int)k, Rr);
    CT_LAUNCH_CHECK();
  }
  {
    LaunchScope ls(K_SPMM, s, 2.0 * nnz * k, 12.0 * nnz + 8.0 * (m + n) * k);
    const unsigned g = (unsigned)((n + 7) / 8 < 65535 ? (n + 7) / 8 : 65535);
    if (k <= 16) k_spmm16<<<g, tb, 0, s>>>(col_ptr, crow, cval, n, Rr, (int)k, Sr);
    else k_spmm<<<g, tb, 0, s>>>(col_ptr, crow, cval, n, Rr, (int)k, Sr);
    CT_LAUNCH_CHECK();
  }
  {
    LaunchScope ls(K_COPY, s, 0.0, 16.0 * n * k);
    k_from_rows<<<dim3((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32)), tb, 0, s>>>(Sr, n, (int)k, S, lds, 0);
    CT_LAUNCH_CHECK();
  }
  return CT_OK;
}

}  // namespace ctqr
