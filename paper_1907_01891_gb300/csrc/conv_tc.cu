// conv_tc.cu -- the surrogate's 32 -> 32 channel 3x3 convolutions (the four
// residual layers, almost all of the network's arithmetic) on the tcgen05
// tensor cores as an implicit GEMM with BF16 operands and FP32 accumulation.
//
// For one image and 128 consecutive output pixels p (row-major, so a tile may
// span image rows):
//   Z[p, o] = sum_{t < 9, c < 32} X[c, p + offset(t)] W[o, c, t]
// is an M = 128, N = 32, K = 288 product.  K is laid out tap-major in five
// 64-element slabs (taps 2s and 2s + 1, 32 channels each; the tenth tap is
// zero), each slab a K-major shared-memory tile with the 128-byte swizzle:
//   A slab: 128 pixel rows x 64 BF16 (the im2col rows, gathered with zero
//           padding at the image border),
//   B slab:  32 output-channel rows x 64 BF16 (the weights).
// One thread issues the 20 tcgen05.mma.kind::f16 (M 128, N 32, K 16) into a
// 32-column TMEM accumulator; the four warps then read their 32 pixel rows
// back with tcgen05.ld and apply bias, ReLU and the residual like the CUDA-core
// kernel (surrogate.cu), storing BF16 NCHW activations.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace ctqr {
namespace {

using namespace tc;

constexpr int kC = 32;                  // channels in and out
constexpr int kM = 128;                 // output pixels per CTA
constexpr int kSlabs = 5;               // 10 taps x 32 channels, 64 per slab
constexpr int kSlabA = kM * 128;        // bytes of one A slab
constexpr int kSlabB = kC * 128;        // bytes of one B slab
constexpr size_t kConvTcSmem = 1024 + (size_t)kSlabs * (kSlabA + kSlabB) + 64;

// Byte offset of the 16-byte chunk q (elements 8q .. 8q+7 of the 64) of row
// `row` in a K-major slab of 128-byte rows with the 128-byte swizzle: 8-row
// groups 1024 bytes apart, the chunk index XORed with the row in the group.
__device__ __forceinline__ uint32_t sw128_chunk(int row, int q) {
  const int r = row & 7;
  return (uint32_t)((row >> 3) * 1024 + r * 128 + ((q ^ r) << 4));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// mode 2 of the CUDA-core kernel: a_out = res + relu(z) (BF16), r_out =
// relu(z) when given; z = conv(in) + bias.
__global__ void __launch_bounds__(128) k_conv_tc(const __nv_bfloat16* __restrict__ in,
                                                 const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
                                                 int H, int W, const __nv_bfloat16* __restrict__ res,
                                                 __nv_bfloat16* __restrict__ r_out, __nv_bfloat16* __restrict__ a_out,
                                                 int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* As = smem;
  unsigned char* Bs = smem + kSlabs * kSlabA;
  uint64_t* done = (uint64_t*)(Bs + kSlabs * kSlabB);
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.y;
  const int64_t plane = (int64_t)H * W;
  const int64_t p0 = (int64_t)blockIdx.x * kM;

  if (tid == 0) {
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(32u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // B: the weights, chunk (o, s, q): taps 2s + q/4, channels (q%4)*8 .. +7
  for (int e = tid; e < kC * kSlabs * 8; e += 128) {
    const int o = e / (kSlabs * 8), sq = e % (kSlabs * 8), s = sq / 8, q = sq % 8;
    const int t = 2 * s + q / 4, c0 = (q % 4) * 8;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (t < 9) {
      const __nv_bfloat16* wp = w + ((size_t)o * kC + c0) * 9 + t;
      v.x = pack2(wp[0], wp[9]);
      v.y = pack2(wp[18], wp[27]);
      v.z = pack2(wp[36], wp[45]);
      v.w = pack2(wp[54], wp[63]);
    }
    *(uint4*)(Bs + s * kSlabB + sw128_chunk(o, q)) = v;
  }
  // A: the im2col rows of this thread's pixel
  {
    const int64_t flat = p0 + tid;
    const bool pix = flat < plane;
    const int y = pix ? (int)(flat / W) : 0, x = pix ? (int)(flat % W) : 0;
    const __nv_bfloat16* ib = in + (size_t)b * kC * plane;
#pragma unroll 1
    for (int s = 0; s < kSlabs; ++s) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int t = 2 * s + q / 4, c0 = (q % 4) * 8;
        const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (pix && t < 9 && yy >= 0 && yy < H && xx >= 0 && xx < W) {
          const __nv_bfloat16* ip = ib + (size_t)c0 * plane + (int64_t)yy * W + xx;
          v.x = pack2(ip[0], ip[plane]);
          v.y = pack2(ip[2 * plane], ip[3 * plane]);
          v.z = pack2(ip[4 * plane], ip[5 * plane]);
          v.w = pack2(ip[6 * plane], ip[7 * plane]);
        }
        *(uint4*)(As + s * kSlabA + sw128_chunk(tid, q)) = v;
      }
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    // M 128, N 32, FP32 accumulator, BF16 A and B, both K-major
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kC >> 3) << 17) |
                           ((uint32_t)(kM >> 4) << 24);
#pragma unroll 1
    for (int s = 0; s < kSlabs; ++s) {
      const uint64_t da = sdesc_sw128(As + s * kSlabA), db = sdesc_sw128(Bs + s * kSlabB);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)  // 16 BF16 = 32 bytes = 2 x 16 B per step
        mma_f16(tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, (s > 0 || kk > 0) ? 1u : 0u);
    }
    mma_commit(done);
  }
  const bool ok = mbar_wait(done, 0u, status, false);
  tc_fence_after();
  if (ok) {
    float acc[kC];
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), acc);
    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16u, acc + 16);
    const int64_t flat = p0 + warp * 32 + lane;
    if (flat < plane) {
#pragma unroll
      for (int o = 0; o < kC; ++o) {
        const size_t idx = ((size_t)b * kC + o) * plane + flat;
        const float z = acc[o] + bias[o];
        const __nv_bfloat16 rb = __float2bfloat16(z > 0.f ? z : 0.f);
        if (r_out) r_out[idx] = rb;
        a_out[idx] = __float2bfloat16(__bfloat162float(res[idx]) + __bfloat162float(rb));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32u) : "memory");
  }
}

}  // namespace

// The residual 32 -> 32 layer a_out = res + relu(conv(in) + bias) for B images
// of H x W on the tensor cores (r_out, when given, keeps relu(conv + bias)).
ct_status launch_conv_tc(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias, int H, int W, int64_t B,
                         const __nv_bfloat16* res, __nv_bfloat16* r_out, __nv_bfloat16* a_out, int* status,
                         cudaStream_t s) {
  if (B <= 0) return CT_OK;
  if (B > 65535) return CT_ERR_INVALID;
  static bool attr = false;
  if (!attr) {
    CT_CUDA_TRY(cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kConvTcSmem));
    attr = true;
  }
  const double px = (double)H * W * B;
  LaunchScope ls(K_CONV, s, 18.0 * px * kC * kC, px * kC * (r_out ? 8.0 : 6.0));
  const dim3 grid((unsigned)(((int64_t)H * W + kM - 1) / kM), (unsigned)B);
  k_conv_tc<<<grid, 128, kConvTcSmem, s>>>(in, w, bias, H, W, res, r_out, a_out, status);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

}  // namespace ctqr
