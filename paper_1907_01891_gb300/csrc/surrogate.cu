// surrogate.cu -- a small convolutional surrogate of the reconstruction and
// the FP64 gate that decides, slice by slice, whether its output is kept or
// the slice is solved through the QR factor (Eq. (qr1)).
//
// Network (NCHW, 3x3 kernels, stride 1, zero padding 1, C = 32, L = 6):
//   a1 = relu(conv0(g'))                       1 -> C
//   a_{l+1} = a_l + relu(conv_l(a_l))          l = 1..L-2, C -> C (residual)
//   y  = conv_{L-1}(a_{L-1})                   C -> 1
// with g' = in_scale * A^T b and x_hat = out_scale * y.  Weights and
// activations are stored in BF16 and every product accumulates in FP32; the
// optimizer keeps FP32 master parameters.  Parameter layout: for each layer
// its weights [out][in][3][3] followed by its biases.
//
// The convolutions tile the image in 16 x 16 output pixels per CTA with the
// 18 x 18 input halo staged in shared memory, input channels in chunks of 8;
// each thread owns one output pixel and all output channels.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "internal.cuh"

namespace ctqr {
namespace {

constexpr int kTile = 16;  // output pixels per CTA side
constexpr int kHalo = kTile + 2;
constexpr int kChunk = 8;  // input channels staged per pass

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// z = conv(in) + bias over one 16 x 16 tile of image blockIdx.z.
// mode 0: y = z (FP32, last layer); mode 1: a = relu(z) (first layer);
// mode 2: a = res + relu(z) (residual layers).  r_out (may be NULL) keeps
// relu(z) in BF16 for the backward pass.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_conv_fwd(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ bias, int H, int W, int mode,
                                                  const __nv_bfloat16* __restrict__ res, __nv_bfloat16* __restrict__ r_out,
                                                  __nv_bfloat16* __restrict__ a_out, float* __restrict__ y_out) {
  constexpr int CC = CIN < kChunk ? CIN : kChunk;
  __shared__ float xs[CC][kHalo][kHalo + 1];
  __shared__ __align__(16) float ws[CC * 9][COUT];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile, b = blockIdx.z;
  const size_t plane = (size_t)H * W;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = bias[o];
  for (int c0 = 0; c0 < CIN; c0 += CC) {
    __syncthreads();
    for (int e = threadIdx.x; e < CC * kHalo * kHalo; e += 256) {
      const int c = e / (kHalo * kHalo), rem = e % (kHalo * kHalo), hy = rem / kHalo, hx = rem % kHalo;
      const int gy = y0 + hy - 1, gx = x0 + hx - 1;
      xs[c][hy][hx] = (gy >= 0 && gy < H && gx >= 0 && gx < W)
                          ? bf(in[((size_t)b * CIN + c0 + c) * plane + (size_t)gy * W + gx])
                          : 0.f;
    }
    for (int e = threadIdx.x; e < CC * 9 * COUT; e += 256) {
      const int o = e % COUT, ck = e / COUT, c = ck / 9, k = ck % 9;
      ws[ck][o] = bf(w[((size_t)o * CIN + c0 + c) * 9 + k]);
    }
    __syncthreads();
    for (int c = 0; c < CC; ++c)
#pragma unroll
      for (int dh = 0; dh < 3; ++dh)
#pragma unroll
        for (int dw = 0; dw < 3; ++dw) {
          const float v = xs[c][ty + dh][tx + dw];
          const float* wr = ws[c * 9 + dh * 3 + dw];
#pragma unroll
          for (int o = 0; o < COUT; ++o) acc[o] = fmaf(wr[o], v, acc[o]);
        }
  }
  const int gy = y0 + ty, gx = x0 + tx;
  if (gy >= H || gx >= W) return;
#pragma unroll
  for (int o = 0; o < COUT; ++o) {
    const size_t idx = ((size_t)b * COUT + o) * plane + (size_t)gy * W + gx;
    if (mode == 0) {
      y_out[idx] = acc[o];
    } else {
      const __nv_bfloat16 rb = __float2bfloat16(acc[o] > 0.f ? acc[o] : 0.f);
      if (r_out) r_out[idx] = rb;
      a_out[idx] = mode == 1 ? rb : __float2bfloat16(bf(res[idx]) + bf(rb));
    }
  }
}

// Gradient with respect to the input of a conv layer: forward y(h, w) uses
// x(h + dh - 1, w + dw - 1), so dx(h, w) = sum_{o,dh,dw} w[o][c][dh][dw] *
// dz(o, h - dh + 1, w - dw + 1).  dx = skip + that (skip may be NULL).
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_conv_bwd_data(const float* __restrict__ dz, const __nv_bfloat16* __restrict__ w,
                                                       int H, int W, const float* __restrict__ skip,
                                                       float* __restrict__ dx) {
  constexpr int OC = COUT < kChunk ? COUT : kChunk;
  __shared__ float zs[OC][kHalo][kHalo + 1];
  __shared__ __align__(16) float ws[OC * 9][CIN];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile, b = blockIdx.z;
  const size_t plane = (size_t)H * W;
  float acc[CIN];
#pragma unroll
  for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
  for (int o0 = 0; o0 < COUT; o0 += OC) {
    __syncthreads();
    for (int e = threadIdx.x; e < OC * kHalo * kHalo; e += 256) {
      const int o = e / (kHalo * kHalo), rem = e % (kHalo * kHalo), hy = rem / kHalo, hx = rem % kHalo;
      const int gy = y0 + hy - 1, gx = x0 + hx - 1;
      zs[o][hy][hx] = (gy >= 0 && gy < H && gx >= 0 && gx < W)
                          ? dz[((size_t)b * COUT + o0 + o) * plane + (size_t)gy * W + gx]
                          : 0.f;
    }
    for (int e = threadIdx.x; e < OC * 9 * CIN; e += 256) {
      const int c = e % CIN, ok = e / CIN, o = ok / 9, k = ok % 9;
      ws[ok][c] = bf(w[((size_t)(o0 + o) * CIN + c) * 9 + k]);
    }
    __syncthreads();
    for (int o = 0; o < OC; ++o)
#pragma unroll
      for (int dh = 0; dh < 3; ++dh)
#pragma unroll
        for (int dw = 0; dw < 3; ++dw) {
          const float v = zs[o][ty + 2 - dh][tx + 2 - dw];
          const float* wr = ws[o * 9 + dh * 3 + dw];
#pragma unroll
          for (int c = 0; c < CIN; ++c) acc[c] = fmaf(wr[c], v, acc[c]);
        }
  }
  const int gy = y0 + ty, gx = x0 + tx;
  if (gy >= H || gx >= W) return;
#pragma unroll
  for (int c = 0; c < CIN; ++c) {
    const size_t idx = ((size_t)b * CIN + c) * plane + (size_t)gy * W + gx;
    dx[idx] = (skip ? skip[idx] : 0.f) + acc[c];
  }
}

// Weight and bias gradients, first stage: CTA (x, y) sums over the tiles
// t = x, x + gridDim.x, ... of the batch, for input channels y*8 .. y*8+7,
// into row x of `part` (entries in the parameter order: weights
// [o][c][3][3] then biases; biases by the y = 0 CTAs).
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) k_conv_bwd_weight(const float* __restrict__ dz, const __nv_bfloat16* __restrict__ in,
                                                         int B, int H, int W, float* __restrict__ part) {
  constexpr int CC = CIN < kChunk ? CIN : kChunk;
  constexpr int NW = COUT * CIN * 9, LEN = NW + COUT;
  constexpr int MINE = COUT * CC * 9 + COUT;  // entries of this CTA (biases only used by y = 0)
  constexpr int PER = (MINE + 255) / 256;
  __shared__ float xs[CC][kHalo][kHalo + 1];
  __shared__ float zs[COUT][kTile * kTile];
  const int c0 = blockIdx.y * CC;
  const int tilesx = (W + kTile - 1) / kTile, tilesy = (H + kTile - 1) / kTile;
  const int ntiles = B * tilesx * tilesy;
  const size_t plane = (size_t)H * W;
  float acc[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) acc[q] = 0.f;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int b = t / (tilesx * tilesy), rem = t % (tilesx * tilesy);
    const int y0 = (rem / tilesx) * kTile, x0 = (rem % tilesx) * kTile;
    __syncthreads();
    for (int e = threadIdx.x; e < CC * kHalo * kHalo; e += 256) {
      const int c = e / (kHalo * kHalo), r2 = e % (kHalo * kHalo), hy = r2 / kHalo, hx = r2 % kHalo;
      const int gy = y0 + hy - 1, gx = x0 + hx - 1;
      xs[c][hy][hx] = (gy >= 0 && gy < H && gx >= 0 && gx < W)
                          ? bf(in[((size_t)b * CIN + c0 + c) * plane + (size_t)gy * W + gx])
                          : 0.f;
    }
    for (int e = threadIdx.x; e < COUT * kTile * kTile; e += 256) {
      const int o = e / (kTile * kTile), p = e % (kTile * kTile);
      const int gy = y0 + p / kTile, gx = x0 + p % kTile;
      zs[o][p] = (gy < H && gx < W) ? dz[((size_t)b * COUT + o) * plane + (size_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + 256 * q;
      if (e < COUT * CC * 9) {
        const int o = e / (CC * 9), c = (e / 9) % CC, k9 = e % 9, dh = k9 / 3, dw = k9 % 3;
        float s = 0.f;
        for (int py = 0; py < kTile; ++py)
#pragma unroll 4
          for (int px = 0; px < kTile; ++px) s = fmaf(zs[o][py * kTile + px], xs[c][py + dh][px + dw], s);
        acc[q] += s;
      } else if (e < MINE && blockIdx.y == 0) {
        const int o = e - COUT * CC * 9;
        float s = 0.f;
        for (int p = 0; p < kTile * kTile; ++p) s += zs[o][p];
        acc[q] += s;
      }
    }
  }
  float* row = part + (size_t)blockIdx.x * LEN;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = threadIdx.x + 256 * q;
    if (e < COUT * CC * 9) {
      const int o = e / (CC * 9), c = (e / 9) % CC, k9 = e % 9;
      row[((size_t)o * CIN + c0 + c) * 9 + k9] = acc[q];
    } else if (e < MINE && blockIdx.y == 0) {
      row[NW + (e - COUT * CC * 9)] = acc[q];
    }
  }
}

// Second stage: add the rows of `part` in order; entries below nw go to gw,
// the rest to gb.
__global__ void k_sum_parts(const float* __restrict__ part, int nparts, int len, int nw, float* __restrict__ gw,
                            float* __restrict__ gb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= len) return;
  float s = 0.f;
  for (int p = 0; p < nparts; ++p) s += part[(size_t)p * len + e];
  if (e < nw) gw[e] = s;
  else gb[e - nw] = s;
}

// dz = da where the stored relu output is positive, else 0.
__global__ void k_relu_grad(const float* __restrict__ da, const __nv_bfloat16* __restrict__ r, size_t n,
                            float* __restrict__ dz) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dz[i] = bf(r[i]) > 0.f ? da[i] : 0.f;
}

// Loss mean((y - t * inv_scale)^2): per-block partial sums (FP64) and the
// gradient dy = 2 (y - t * inv_scale) / n.
__global__ void k_mse(const float* __restrict__ y, const double* __restrict__ t, double inv_scale, size_t n,
                      float* __restrict__ dy, double* __restrict__ part) {
  __shared__ double sh[8];
  double s = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double d = (double)y[i] - t[i] * inv_scale;
    s += d * d;
    dy[i] = (float)(2.0 * d / (double)n);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += sh[q];
    part[blockIdx.x] = tot / (double)n;
  }
}

// Adam on the FP32 parameters (bias-corrected with c1 = 1 - b1^t,
// c2 = 1 - b2^t); refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       __nv_bfloat16* __restrict__ pb, int n, float lr, float b1, float b2, float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  pb[i] = __float2bfloat16(pi);
}

__global__ void k_f64_to_bf16(const double* __restrict__ x, double scale, size_t n, __nv_bfloat16* __restrict__ y) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16((float)(x[i] * scale));
}

__global__ void k_f32_to_f64(const float* __restrict__ x, double scale, size_t n, double* __restrict__ y) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (double)x[i] * scale;
}

__global__ void k_f32_to_bf16(const float* __restrict__ x, size_t n, __nv_bfloat16* __restrict__ y) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// Uniform(-a, a) initialisation from the splitmix64 hash of (seed, index).
__global__ void k_init_uniform(float* __restrict__ p, int n, float a, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const float u = (float)((double)(z >> 40) * (1.0 / 16777216.0));
  p[i] = a * (2.f * u - 1.f);
}

// Gate: resid[c] = sqrt(rn2[c] / bn2[c]) (sqrt(rn2[c]) when bn2[c] = 0);
// slices with resid <= tol pass (NaN fails).  One warp compacts the failing
// slice indices in increasing order into idx[0:*nfail] and writes the
// largest passing residual to *max_pass.
__global__ void k_gate(const double* __restrict__ rn2, const double* __restrict__ bn2, int k, double tol,
                       double* __restrict__ resid, int* __restrict__ idx, int* __restrict__ nfail,
                       double* __restrict__ max_pass) {
  const int lane = threadIdx.x;
  int count = 0;
  double mx = 0.0;
  for (int c0 = 0; c0 < k; c0 += 32) {
    const int c = c0 + lane;
    bool fail = false;
    if (c < k) {
      const double r = bn2[c] > 0.0 ? sqrt(rn2[c] / bn2[c]) : sqrt(rn2[c]);
      if (resid) resid[c] = r;
      fail = !(r <= tol);
      if (!fail) mx = fmax(mx, r);
    }
    const unsigned ball = __ballot_sync(0xffffffffu, fail);
    if (fail) idx[count + __popc(ball & ((1u << lane) - 1u))] = c;
    count += __popc(ball);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    *nfail = count;
    *max_pass = mx;
  }
}

// dst[r, j] = src[r, idx[j]] for r < rows_src, 0 for rows_src <= r < rows.
__global__ void k_gather_cols(const double* __restrict__ src, int64_t lds, int64_t rows_src, const int* __restrict__ idx,
                              int64_t rows, double* __restrict__ dst, int64_t ldd) {
  const int j = blockIdx.y;
  const double* s = src + (size_t)idx[j] * lds;
  double* d = dst + (size_t)j * ldd;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
    d[r] = r < rows_src ? s[r] : 0.0;
}

// dst[r, idx[j]] = src[r, j].
__global__ void k_scatter_cols(const double* __restrict__ src, int64_t lds, const int* __restrict__ idx, int64_t rows,
                               double* __restrict__ dst, int64_t ldd) {
  const int j = blockIdx.y;
  const double* s = src + (size_t)j * lds;
  double* d = dst + (size_t)idx[j] * ldd;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
    d[r] = s[r];
}

unsigned blocks_for(size_t n) {
  const size_t b = (n + 255) / 256;
  return (unsigned)(b == 0 ? 1 : (b < 4096 ? b : 4096));
}

}  // namespace

// ----------------------------------------------------------------- the model
struct Surrogate {
  static constexpr int C = 32;
  static constexpr int L = 6;
  static constexpr int kPartRows = 512;  // CTAs of the weight-gradient first stage
  static constexpr int kMaxBatch = 256;  // images per network launch
  static int cin(int l) { return l == 0 ? 1 : C; }
  static int cout(int l) { return l == L - 1 ? 1 : C; }

  ct_geometry geom{};
  int nx = 0, ny = 0;
  int64_t m = 0, n = 0;
  double in_scale = 1.0, out_scale = 1.0;
  int w_off[L] = {}, b_off[L] = {}, nparam = 0;
  float *p = nullptr, *g = nullptr, *mom = nullptr, *vel = nullptr, *part = nullptr;
  __nv_bfloat16* pb = nullptr;
  int64_t step = 0;
  int64_t cap = 0;                       // images the activation buffers hold
  __nv_bfloat16 *a[L] = {}, *r[L] = {};  // a[0] = scaled input; r[l] = relu output feeding a[l]
  float *y = nullptr, *dy = nullptr, *dA = nullptr, *dA2 = nullptr, *dZ = nullptr;
  double* loss_part = nullptr;
  SparseSystem sp;
  int* status = nullptr;  // sparse build status word
  // gate scratch
  double *rn2 = nullptr, *bn2 = nullptr, *Rbuf = nullptr, *max_pass = nullptr;
  int *fail_idx = nullptr, *nfail = nullptr;

  ~Surrogate() { release(); }
  void release_acts() {
    for (int l = 0; l < L; ++l) {
      if (a[l]) cudaFree(a[l]);
      if (r[l]) cudaFree(r[l]);
      a[l] = r[l] = nullptr;
    }
    for (float* q : {y, dy, dA, dA2, dZ})
      if (q) cudaFree(q);
    y = dy = dA = dA2 = dZ = nullptr;
    cap = 0;
  }
  void release() {
    release_acts();
    for (float* q : {p, g, mom, vel, part})
      if (q) cudaFree(q);
    p = g = mom = vel = part = nullptr;
    for (void* q : {(void*)pb, (void*)loss_part, (void*)status, (void*)rn2, (void*)bn2, (void*)Rbuf,
                    (void*)max_pass, (void*)fail_idx, (void*)nfail})
      if (q) cudaFree(q);
    pb = nullptr;
    loss_part = rn2 = bn2 = Rbuf = max_pass = nullptr;
    status = fail_idx = nfail = nullptr;
    sp.release();
  }
  ct_status ensure(int64_t batch) {
    if (batch <= cap) return CT_OK;
    release_acts();
    const size_t plane = (size_t)nx * ny;
    for (int l = 0; l < L; ++l) {
      const size_t ch = l == 0 ? 1 : C;
      CT_CUDA_TRY(cudaMalloc(&a[l], batch * ch * plane * sizeof(__nv_bfloat16)));
      if (l > 0) CT_CUDA_TRY(cudaMalloc(&r[l], batch * ch * plane * sizeof(__nv_bfloat16)));
    }
    CT_CUDA_TRY(cudaMalloc(&y, batch * plane * sizeof(float)));
    CT_CUDA_TRY(cudaMalloc(&dy, batch * plane * sizeof(float)));
    CT_CUDA_TRY(cudaMalloc(&dA, batch * C * plane * sizeof(float)));
    CT_CUDA_TRY(cudaMalloc(&dA2, batch * C * plane * sizeof(float)));
    CT_CUDA_TRY(cudaMalloc(&dZ, batch * C * plane * sizeof(float)));
    cap = batch;
    return CT_OK;
  }
};

namespace {

// The residual layers' forward convolutions run on the tensor cores unless
// CTQR_CONV_SIMT=1 selects the CUDA-core kernel (for comparison).
bool conv_tc_enabled() {
  static const bool on = [] {
    const char* e = getenv("CTQR_CONV_SIMT");
    return !(e && *e == '1');
  }();
  return on;
}

dim3 conv_grid(const Surrogate& s, int64_t B) {
  return dim3((unsigned)((s.nx + kTile - 1) / kTile), (unsigned)((s.ny + kTile - 1) / kTile), (unsigned)B);
}

// Network forward for B images whose scaled input is in a[0]; y = output.
// train keeps the relu outputs for the backward pass.
ct_status forward(Surrogate& s, int64_t B, bool train, cudaStream_t st) {
  constexpr int C = Surrogate::C, L = Surrogate::L;
  const dim3 grid = conv_grid(s, B);
  const double px = (double)s.nx * s.ny * B;
  {
    LaunchScope ls(K_CONV, st, 18.0 * px * C, px * (2.0 + (train ? 4.0 : 2.0) * C));
    k_conv_fwd<1, C><<<grid, 256, 0, st>>>(s.a[0], s.pb + s.w_off[0], s.p + s.b_off[0], s.ny, s.nx, 1, nullptr,
                                           train ? s.r[1] : nullptr, s.a[1], nullptr);
  }
  for (int l = 1; l < L - 1; ++l) {
    if (conv_tc_enabled()) {
      // the 32 -> 32 residual layers on the tensor cores (conv_tc.cu)
      const ct_status r = launch_conv_tc(s.a[l], s.pb + s.w_off[l], s.p + s.b_off[l], s.ny, s.nx, B, s.a[l],
                                         train ? s.r[l + 1] : nullptr, s.a[l + 1], s.status, st);
      if (r != CT_OK) return r;
      continue;
    }
    LaunchScope ls(K_CONV, st, 18.0 * px * C * C, px * C * (train ? 8.0 : 6.0));
    k_conv_fwd<C, C><<<grid, 256, 0, st>>>(s.a[l], s.pb + s.w_off[l], s.p + s.b_off[l], s.ny, s.nx, 2, s.a[l],
                                           train ? s.r[l + 1] : nullptr, s.a[l + 1], nullptr);
  }
  {
    LaunchScope ls(K_CONV, st, 18.0 * px * C, px * (2.0 * C + 4.0));
    k_conv_fwd<C, 1><<<grid, 256, 0, st>>>(s.a[L - 1], s.pb + s.w_off[L - 1], s.p + s.b_off[L - 1], s.ny, s.nx, 0,
                                           nullptr, nullptr, nullptr, s.y);
  }
  CT_LAUNCH_CHECK();
  return CT_OK;
}

template <int CIN, int COUT>
ct_status weight_grad(Surrogate& s, int layer, const float* dz, const __nv_bfloat16* in, int64_t B, cudaStream_t st) {
  constexpr int CC = CIN < kChunk ? CIN : kChunk;
  constexpr int NW = COUT * CIN * 9, LEN = NW + COUT;
  const int64_t tiles = B * ((s.nx + kTile - 1) / kTile) * ((s.ny + kTile - 1) / kTile);
  const int rows = (int)std::min<int64_t>(tiles, Surrogate::kPartRows);
  const double px = (double)s.nx * s.ny * B;
  {
    LaunchScope ls(K_CONV, st, 18.0 * px * CIN * COUT, px * (2.0 * CIN + 4.0 * COUT) + 4.0 * rows * LEN);
    k_conv_bwd_weight<CIN, COUT><<<dim3(rows, CIN / CC), 256, 0, st>>>(dz, in, (int)B, s.ny, s.nx, s.part);
  }
  LaunchScope ls(K_CONV, st, (double)rows * LEN, 4.0 * rows * LEN);
  k_sum_parts<<<(LEN + 255) / 256, 256, 0, st>>>(s.part, rows, LEN, NW, s.g + s.w_off[layer], s.g + s.b_off[layer]);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

// Backward pass from dy to every parameter gradient (g).
ct_status backward(Surrogate& s, int64_t B, cudaStream_t st) {
  constexpr int C = Surrogate::C, L = Surrogate::L;
  const dim3 grid = conv_grid(s, B);
  const size_t act = (size_t)B * C * s.nx * s.ny;
  const double px = (double)s.nx * s.ny * B;
  ct_status r;
  if ((r = weight_grad<C, 1>(s, L - 1, s.dy, s.a[L - 1], B, st)) != CT_OK) return r;
  {
    LaunchScope ls(K_CONV, st, 18.0 * px * C, px * (4.0 + 4.0 * C));
    k_conv_bwd_data<C, 1><<<grid, 256, 0, st>>>(s.dy, s.pb + s.w_off[L - 1], s.ny, s.nx, nullptr, s.dA);
  }
  // layer l maps a[l] to a[l+1] = a[l] + r[l+1]: d a[l] = d a[l+1] + conv_l^T (d a[l+1] * [r[l+1] > 0])
  for (int l = L - 2; l >= 1; --l) {
    {
      LaunchScope ls(K_CONV, st, 0.0, 10.0 * act);
      k_relu_grad<<<blocks_for(act), 256, 0, st>>>(s.dA, s.r[l + 1], act, s.dZ);
    }
    if ((r = weight_grad<C, C>(s, l, s.dZ, s.a[l], B, st)) != CT_OK) return r;
    {
      LaunchScope ls(K_CONV, st, 18.0 * px * C * C, 12.0 * act);
      k_conv_bwd_data<C, C><<<grid, 256, 0, st>>>(s.dZ, s.pb + s.w_off[l], s.ny, s.nx, s.dA, s.dA2);
    }
    std::swap(s.dA, s.dA2);
  }
  {
    LaunchScope ls(K_CONV, st, 0.0, 10.0 * act);
    k_relu_grad<<<blocks_for(act), 256, 0, st>>>(s.dA, s.r[1], act, s.dZ);
  }
  if ((r = weight_grad<1, C>(s, 0, s.dZ, s.a[0], B, st)) != CT_OK) return r;
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status load_inputs(Surrogate& s, const double* G, int64_t B, cudaStream_t st) {
  const size_t n = (size_t)B * s.nx * s.ny;
  LaunchScope ls(K_CONV, st, (double)n, 10.0 * n);
  k_f64_to_bf16<<<blocks_for(n), 256, 0, st>>>(G, s.in_scale, n, s.a[0]);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

// Loss (and dy) of the batch in y against targets X; the partial sums stay
// on the device in loss_part[0:nb).
ct_status mse(Surrogate& s, const double* X, int64_t B, unsigned* nb_out, cudaStream_t st) {
  const size_t n = (size_t)B * s.nx * s.ny;
  const unsigned nb = std::min(blocks_for(n), 1024u);
  LaunchScope ls(K_CONV, st, 4.0 * n, 16.0 * n);
  k_mse<<<nb, 256, 0, st>>>(s.y, X, 1.0 / s.out_scale, n, s.dy, s.loss_part);
  CT_LAUNCH_CHECK();
  *nb_out = nb;
  return CT_OK;
}

ct_status read_loss(Surrogate& s, unsigned nb, double* loss, cudaStream_t st) {
  std::vector<double> h(nb);
  CT_CUDA_TRY(cudaMemcpyAsync(h.data(), s.loss_part, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  CT_CUDA_TRY(cudaStreamSynchronize(st));
  double tot = 0.0;
  for (double v : h) tot += v;
  *loss = tot;
  return CT_OK;
}

// x_hat = out_scale * network(in_scale * G) for k images, kMaxBatch at a time.
ct_status run_network(Surrogate& s, const double* G, double* Xhat, int64_t ldx, int64_t k, cudaStream_t st) {
  const size_t plane = (size_t)s.nx * s.ny;
  ct_status r;
  for (int64_t b0 = 0; b0 < k; b0 += Surrogate::kMaxBatch) {
    const int64_t nb = std::min<int64_t>(Surrogate::kMaxBatch, k - b0);
    if ((r = s.ensure(nb)) != CT_OK) return r;
    if ((r = load_inputs(s, G + b0 * plane, nb, st)) != CT_OK) return r;
    if ((r = forward(s, nb, false, st)) != CT_OK) return r;
    if (ldx == (int64_t)plane) {
      LaunchScope ls(K_CONV, st, (double)nb * plane, 12.0 * nb * plane);
      k_f32_to_f64<<<blocks_for(nb * plane), 256, 0, st>>>(s.y, s.out_scale, nb * plane, Xhat + b0 * ldx);
      CT_LAUNCH_CHECK();
    } else {
      for (int64_t j = 0; j < nb; ++j) {
        LaunchScope ls(K_CONV, st, (double)plane, 12.0 * plane);
        k_f32_to_f64<<<blocks_for(plane), 256, 0, st>>>(s.y + j * plane, s.out_scale, plane, Xhat + (b0 + j) * ldx);
        CT_LAUNCH_CHECK();
      }
    }
  }
  return CT_OK;
}

bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

}  // namespace
}  // namespace ctqr

using namespace ctqr;

struct ct_surrogate {
  Surrogate s;
};

extern "C" {

ct_status ct_surrogate_init(const ct_geometry* g, const ct_surrogate_opts* opts, ct_surrogate** out) {
  if (!g || !out) return CT_ERR_INVALID;
  *out = nullptr;
  int64_t m = 0, n = 0;
  ct_status st = ct_system_size(g, 0.0, &m, &n);
  if (st != CT_OK) return st;
  if (opts && !(opts->in_scale > 0.0 && opts->out_scale > 0.0)) return CT_ERR_INVALID;
  ct_surrogate* h = new ct_surrogate;
  Surrogate& s = h->s;
  s.geom = *g;
  s.nx = g->nx;
  s.ny = g->ny;
  s.m = m;
  s.n = n;
  s.in_scale = opts ? opts->in_scale : 1.0;
  s.out_scale = opts ? opts->out_scale : 1.0;
  const uint64_t seed = opts ? opts->seed : 0;
  int off = 0;
  for (int l = 0; l < Surrogate::L; ++l) {
    s.w_off[l] = off;
    off += Surrogate::cout(l) * Surrogate::cin(l) * 9;
    s.b_off[l] = off;
    off += Surrogate::cout(l);
  }
  s.nparam = off;
  const int maxlen = Surrogate::C * Surrogate::C * 9 + Surrogate::C;
  auto fail = [&](ct_status e) {
    cudaGetLastError();
    delete h;
    return e;
  };
  if (cudaMalloc(&s.p, off * sizeof(float)) != cudaSuccess || cudaMalloc(&s.g, off * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&s.mom, off * sizeof(float)) != cudaSuccess || cudaMalloc(&s.vel, off * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&s.pb, off * sizeof(__nv_bfloat16)) != cudaSuccess ||
      cudaMalloc(&s.part, (size_t)Surrogate::kPartRows * maxlen * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&s.loss_part, 1024 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&s.status, sizeof(int)) != cudaSuccess)
    return fail(CT_ERR_NOMEM);
  cudaStream_t st0 = 0;
  if (cudaMemsetAsync(s.mom, 0, off * sizeof(float), st0) != cudaSuccess ||
      cudaMemsetAsync(s.vel, 0, off * sizeof(float), st0) != cudaSuccess ||
      cudaMemsetAsync(s.p, 0, off * sizeof(float), st0) != cudaSuccess ||
      cudaMemsetAsync(s.status, 0, sizeof(int), st0) != cudaSuccess)
    return fail(CT_ERR_CUDA);
  for (int l = 0; l < Surrogate::L; ++l) {
    // uniform bound sqrt(6 / fan_in); the output layer starts 10x smaller; biases 0
    const int len = Surrogate::cout(l) * Surrogate::cin(l) * 9;
    const float a = sqrtf(6.f / (9.f * Surrogate::cin(l))) * (l == Surrogate::L - 1 ? 0.1f : 1.f);
    k_init_uniform<<<(len + 255) / 256, 256, 0, st0>>>(s.p + s.w_off[l], len, a, seed * 1000003ull + (uint64_t)l);
  }
  k_f32_to_bf16<<<blocks_for(off), 256, 0, st0>>>(s.p, off, s.pb);
  if (cudaGetLastError() != cudaSuccess) return fail(CT_ERR_CUDA);
  if ((st = s.sp.build(g, Surrogate::kMaxBatch, s.status, st0)) != CT_OK) return fail(st);
  int hs = 0;
  if (cudaMemcpy(&hs, s.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return fail(CT_ERR_CUDA);
  if (hs != 0) return fail((ct_status)hs);
  *out = h;
  return CT_OK;
}

int64_t ct_surrogate_num_params(const ct_surrogate* h) { return h ? h->s.nparam : 0; }

ct_status ct_surrogate_params(ct_surrogate* h, float* host, int set) {
  if (!h || !host) return CT_ERR_INVALID;
  Surrogate& s = h->s;
  if (set) {
    CT_CUDA_TRY(cudaMemcpy(s.p, host, s.nparam * sizeof(float), cudaMemcpyHostToDevice));
    k_f32_to_bf16<<<blocks_for(s.nparam), 256>>>(s.p, s.nparam, s.pb);
    CT_LAUNCH_CHECK();
    CT_CUDA_TRY(cudaDeviceSynchronize());
  } else {
    CT_CUDA_TRY(cudaMemcpy(host, s.p, s.nparam * sizeof(float), cudaMemcpyDeviceToHost));
  }
  return CT_OK;
}

ct_status ct_surrogate_backproject(ct_surrogate* h, const double* B, int64_t ldb, int64_t k, double* G, void* stream) {
  if (!h || k < 0) return CT_ERR_INVALID;
  Surrogate& s = h->s;
  if (k == 0) return CT_OK;
  if (!B || !G || ldb < s.m || !aligned8(B) || !aligned8(G)) return CT_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  for (int64_t c0 = 0; c0 < k; c0 += Surrogate::kMaxBatch) {
    const int64_t kc = std::min<int64_t>(Surrogate::kMaxBatch, k - c0);
    ct_status r = s.sp.apply_t(B + c0 * ldb, ldb, kc, G + c0 * s.n, s.n, st);
    if (r != CT_OK) return r;
  }
  return CT_OK;
}

ct_status ct_surrogate_project(ct_surrogate* h, const double* X, int64_t k, double* B, int64_t ldb, void* stream) {
  if (!h || k < 0) return CT_ERR_INVALID;
  Surrogate& s = h->s;
  if (k == 0) return CT_OK;
  if (!B || !X || ldb < s.m || !aligned8(B) || !aligned8(X)) return CT_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  for (int64_t c0 = 0; c0 < k; c0 += Surrogate::kMaxBatch) {
    const int64_t kc = std::min<int64_t>(Surrogate::kMaxBatch, k - c0);
    ct_status r = s.sp.apply(X + c0 * s.n, s.n, kc, B + c0 * ldb, ldb, 0, st);
    if (r != CT_OK) return r;
  }
  return CT_OK;
}

ct_status ct_surrogate_train_step(ct_surrogate* h, const double* G, const double* X, int64_t batch, float lr,
                                  double* loss, void* stream) {
  if (!h || !G || !X || batch <= 0 || batch > 65535 || !(lr >= 0.f)) return CT_ERR_INVALID;
  Surrogate& s = h->s;
  cudaStream_t st = (cudaStream_t)stream;
  ct_status r;
  unsigned nb = 0;
  if ((r = s.ensure(batch)) != CT_OK) return r;
  if ((r = load_inputs(s, G, batch, st)) != CT_OK) return r;
  if ((r = forward(s, batch, true, st)) != CT_OK) return r;
  if ((r = mse(s, X, batch, &nb, st)) != CT_OK) return r;
  if ((r = backward(s, batch, st)) != CT_OK) return r;
  s.step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)s.step), c2 = 1.f - powf(b2, (float)s.step);
  {
    LaunchScope ls(K_CONV, st, 12.0 * s.nparam, 30.0 * s.nparam);
    k_adam<<<(s.nparam + 255) / 256, 256, 0, st>>>(s.p, s.mom, s.vel, s.g, s.pb, s.nparam, lr, b1, b2, c1, c2, 1e-8f);
  }
  CT_LAUNCH_CHECK();
  if (loss) return read_loss(s, nb, loss, st);
  return CT_OK;
}

ct_status ct_surrogate_grad(ct_surrogate* h, const double* G, const double* X, int64_t batch, double* loss,
                            float* grad_host, void* stream) {
  if (!h || !G || !X || batch <= 0 || batch > 65535) return CT_ERR_INVALID;
  Surrogate& s = h->s;
  cudaStream_t st = (cudaStream_t)stream;
  ct_status r;
  unsigned nb = 0;
  if ((r = s.ensure(batch)) != CT_OK) return r;
  if ((r = load_inputs(s, G, batch, st)) != CT_OK) return r;
  if ((r = forward(s, batch, true, st)) != CT_OK) return r;
  if ((r = mse(s, X, batch, &nb, st)) != CT_OK) return r;
  if ((r = backward(s, batch, st)) != CT_OK) return r;
  if (grad_host) CT_CUDA_TRY(cudaMemcpyAsync(grad_host, s.g, s.nparam * sizeof(float), cudaMemcpyDeviceToHost, st));
  double l = 0.0;
  if ((r = read_loss(s, nb, &l, st)) != CT_OK) return r;
  if (loss) *loss = l;
  return CT_OK;
}

ct_status ct_surrogate_forward(ct_surrogate* h, const double* G, double* Xhat, int64_t k, void* stream) {
  if (!h || k < 0) return CT_ERR_INVALID;
  if (k == 0) return CT_OK;
  if (!G || !Xhat) return CT_ERR_INVALID;
  return run_network(h->s, G, Xhat, h->s.n, k, (cudaStream_t)stream);
}

ct_status ct_surrogate_infer(ct_surrogate* h, const double* B, int64_t ldb, double* X, int64_t ldx, int64_t k,
                             double tol, const ct_factor* f, const ct_refine_opts* ropts, double* resid,
                             ct_surrogate_report* report, void* stream) {
  const auto t0 = std::chrono::steady_clock::now();
  if (report) memset(report, 0, sizeof(*report));
  if (!h || k < 0 || !(tol >= 0.0)) return CT_ERR_INVALID;
  if (k == 0) return CT_OK;
  Surrogate& s = h->s;
  if (!B || !X || ldb < s.m || ldx < s.n || !aligned8(B) || !aligned8(X) || k > INT32_MAX) return CT_ERR_INVALID;
  if (f) {
    // f factors A (f->m = rays) or [A; lambda I] (f->m = rays + n, lambda in ropts)
    const bool stacked = ropts && ropts->lambda > 0.0;
    if (f->n != s.n || f->m != (stacked ? s.m + s.n : s.m)) return CT_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t KB = Surrogate::kMaxBatch;
  if (!s.rn2) {
    CT_CUDA_TRY(cudaMalloc(&s.rn2, KB * sizeof(double)));
    CT_CUDA_TRY(cudaMalloc(&s.bn2, KB * sizeof(double)));
    CT_CUDA_TRY(cudaMalloc(&s.Rbuf, (size_t)s.m * KB * sizeof(double)));
    CT_CUDA_TRY(cudaMalloc(&s.max_pass, sizeof(double)));
    CT_CUDA_TRY(cudaMalloc(&s.fail_idx, KB * sizeof(int)));
    CT_CUDA_TRY(cudaMalloc(&s.nfail, sizeof(int)));
  }
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  struct EvFree {
    cudaEvent_t* e;
    ~EvFree() { for (int i = 0; i < 4; ++i) if (e[i]) cudaEventDestroy(e[i]); }
  } evfree{ev};
  for (auto& e : ev) CT_CUDA_TRY(cudaEventCreate(&e));
  double ms_net = 0.0, ms_gate = 0.0, ms_fb = 0.0, max_res = 0.0;
  int64_t fallbacks = 0;
  ct_status result = CT_OK;
  // G: backprojections of one chunk; afterwards the fallback's compacted
  // right-hand sides (ldf x nf) and solutions (n x nf)
  const int64_t ldf = f ? (f->m + 1) / 2 * 2 : 0;
  const size_t gsz = std::max((size_t)s.n * KB, (size_t)(ldf + s.n) * KB);
  double* G = nullptr;
  CT_CUDA_TRY(cudaMallocAsync((void**)&G, gsz * sizeof(double), st));
  struct GFree { double* p; cudaStream_t s; ~GFree() { cudaFreeAsync(p, s); } } gfree{G, st};
  for (int64_t c0 = 0; c0 < k && result == CT_OK; c0 += KB) {
    const int64_t kc = std::min<int64_t>(KB, k - c0);
    const double* Bc = B + c0 * ldb;
    double* Xc = X + c0 * ldx;
    ct_status r;
    CT_CUDA_TRY(cudaEventRecord(ev[0], st));
    if ((r = s.sp.apply_t(Bc, ldb, kc, G, s.n, st)) != CT_OK) return r;
    if ((r = run_network(s, G, Xc, ldx, kc, st)) != CT_OK) return r;
    CT_CUDA_TRY(cudaEventRecord(ev[1], st));
    // gate: R = B - A x_hat with the exact FP64 A, per-slice norms, compaction
    if ((r = launch_copy_matrix(Bc, CT_F64, ldb, s.Rbuf, CT_F64, s.m, s.m, kc, st)) != CT_OK) return r;
    if ((r = s.sp.apply(Xc, ldx, kc, s.Rbuf, s.m, 1, st)) != CT_OK) return r;
    if ((r = launch_col_norms2(s.Rbuf, s.m, s.m, kc, s.rn2, st)) != CT_OK) return r;
    if ((r = launch_col_norms2(Bc, ldb, s.m, kc, s.bn2, st)) != CT_OK) return r;
    {
      LaunchScope ls(K_GATE, st, 4.0 * kc, 24.0 * kc);
      k_gate<<<1, 32, 0, st>>>(s.rn2, s.bn2, (int)kc, tol, resid ? resid + c0 : nullptr, s.fail_idx, s.nfail,
                               s.max_pass);
      CT_LAUNCH_CHECK();
    }
    CT_CUDA_TRY(cudaEventRecord(ev[2], st));
    int nf = 0;
    double mp = 0.0;
    CT_CUDA_TRY(cudaMemcpyAsync(&nf, s.nfail, sizeof(int), cudaMemcpyDeviceToHost, st));
    CT_CUDA_TRY(cudaMemcpyAsync(&mp, s.max_pass, sizeof(double), cudaMemcpyDeviceToHost, st));
    CT_CUDA_TRY(cudaStreamSynchronize(st));
    fallbacks += nf;
    max_res = std::max(max_res, mp);
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ev[0], ev[1]) == cudaSuccess) ms_net += t;
    if (cudaEventElapsedTime(&t, ev[1], ev[2]) == cudaSuccess) ms_gate += t;
    if (nf > 0 && f) {
      // compact the failing sinograms (rows past the rays are the zero
      // right-hand side of the lambda*I rows), solve through the factor,
      // scatter the solutions back
      double* Bf = G;
      double* Xf = G + (size_t)ldf * nf;
      CT_CUDA_TRY(cudaEventRecord(ev[2], st));
      {
        LaunchScope ls(K_GATE, st, 0.0, 16.0 * f->m * nf);
        k_gather_cols<<<dim3(std::max(1u, std::min(64u, (unsigned)((f->m + 255) / 256))), nf), 256, 0, st>>>(
            Bc, ldb, s.m, s.fail_idx, f->m, Bf, ldf);
        CT_LAUNCH_CHECK();
      }
      const bool mixed = f->prec != CT_PREC_F64;
      ct_report rep;
      r = reconstruct_with(f, mixed ? &s.sp : nullptr, Bf, ldf, Xf, s.n, nf, ropts, &rep, st);
      if (r != CT_OK) {
        result = r;
      } else {
        LaunchScope ls(K_GATE, st, 0.0, 16.0 * s.n * nf);
        k_scatter_cols<<<dim3(std::max(1u, std::min(64u, (unsigned)((s.n + 255) / 256))), nf), 256, 0, st>>>(
            Xf, s.n, s.fail_idx, s.n, Xc, ldx);
        CT_LAUNCH_CHECK();
      }
      CT_CUDA_TRY(cudaEventRecord(ev[3], st));
      CT_CUDA_TRY(cudaEventSynchronize(ev[3]));
      if (cudaEventElapsedTime(&t, ev[2], ev[3]) == cudaSuccess) ms_fb += t;
    }
  }
  if (report) {
    report->slices = k;
    report->fallbacks = fallbacks;
    report->max_residual = max_res;
    report->ms_network = ms_net;
    report->ms_gate = ms_gate;
    report->ms_fallback = ms_fb;
    report->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return result;
}

void ct_surrogate_destroy(ct_surrogate* h) { delete h; }

}  // extern "C"
