// tc_f16.cu -- tensor-core products of the mixed-precision trailing update
// with every FP32 operand split into two FP16 parts.
//
// An FP32 value x, scaled by a power of two s so that |x s| < 2^15, is held
// as h + l with h = fp16(x s) and l = fp16(x s - h): h carries the leading 11
// significant bits and l the next 11, so h + l keeps x to about 2^-22
// relatively (an element whose l falls below FP16's normal range keeps an
// absolute 2^-25 / s instead).  A product of two such operands takes three
// FP16 tensor-core products with FP32 accumulation,
//     (h_a + l_a)(h_b + l_b) ~ h_a h_b + l_a h_b + h_a l_b
// (the dropped l_a l_b is ~2^-22 of the product), and the epilogue multiplies
// by 1 / (s_a s_b), a power of two.  tcgen05.mma.kind::f16 runs at twice the
// TF32 rate on operands of half the size, so this takes half the tensor time
// and half the operand bytes of the three-pass TF32 split (tc_gemm.cu) for
// about the same accuracy.  The scales: reflectors V by the fixed 2^kVExp16
// (|v| is about 1 or less, checked when V is split); the trailing matrix and
// W' = T^T V^T C per column, from a bound on the column's largest magnitude
// (its 2-norm for the trailing matrix, its maximum for W'), so that small
// columns keep their relative accuracy.
//
// Kernels (one CTA per SM or a grid over output tiles; every wait bounded):
//   k_tc_gemm16    W (M x N) = A^T B over the K range of split z (blockIdx.z),
//                  A (K x M) pre-split, MT = 1 or 2 M tiles of 128 per CTA
//                  (two TMEM accumulators sharing each B slice, so B is read
//                  once for up to 256 reflectors).  B (K x N) is either
//                  pre-split or FP32, split in shared memory by four converter
//                  warps with its per-column scale into a two-slot ring beside
//                  the TMA ring.  K slices of 32 elements (64-byte rows,
//                  64-byte swizzle), TMEM accumulation
//                  restarted every 256 rows and the chunks summed on the CUDA
//                  cores (the tensor cores' FP32 sums truncate) by drain
//                  warps, two warpgroups per M tile when B is raw.
//   k_tc_update16  C (M x N) -= A^T B with both operands pre-split, K <= 256:
//                  persistent, warp-specialised, double-buffered TMEM, C
//                  prefetched by the epilogue warps; per-column inverse
//                  scales.  K slices of 64 elements (128-byte swizzle) in two
//                  64 KB stages beside a 64 KB buffer for the next tile's C.
#include <cuda.h>
#include <cuda_fp16.h>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace ctqr {

namespace {

using namespace tc;

constexpr int kBM = 128;
constexpr int kBN = 128;
constexpr int kBK = 32;                               // FP16 elements per K slice of k_tc_gemm16
constexpr uint32_t kT16 = kBM * kBK * 2;              // 8 KB: a 128 x 32 FP16 tile
constexpr uint32_t kTRaw = kBN * kBK * 4;             // 16 KB: a 128 x 32 FP32 tile
constexpr int kChunkSlices = 8;                       // 256 K rows per TMEM chunk
constexpr int kUK = 64;                               // FP16 elements per K slice of k_tc_update16
constexpr uint32_t kUTile = kBM * kUK * 2;            // 16 KB: a 128 x 64 FP16 tile (128-byte rows)
constexpr int kUStages = 2;                           // 2 x 64 KB operand stages beside the 64 KB C buffer
constexpr int kUpdThreads = 384;
constexpr size_t kUpdCbufBytes = (size_t)256 * 64 * sizeof(float);

__device__ __forceinline__ float split16(float x, float s, __half& h, __half& l) {
  const float xs = x * s;
  h = __float2half_rn(xs);
  l = __float2half_rn(xs - __half2float(h));
  return xs;
}

// Eight consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// Shared-memory matrix descriptor: K-major tile with 64-byte rows, 64-byte
// swizzle, 8-row groups 512 bytes apart (SBO), fixed field 0b001 at bit 46,
// layout type 4 (SWIZZLE_64B) in bits 61-63.
__device__ __forceinline__ uint64_t sdesc_sw64(const void* p) {
  const uint64_t a = smem_u32(p);
  uint64_t d = (a >> 4) & 0x3FFFull;
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

__device__ __forceinline__ void mma_f16_ss(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                           uint32_t accum) {
  mma_f16(d_tmem, a, b, idesc, accum);
}

// Instruction descriptor of kind::f16 with FP16 A and B, FP32 D, both
// operands K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_f16(int n) {
  return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

struct G16Args {
  int64_t M, N, K;
  int64_t k_chunk;          // K rows per split (multiple of kBK)
  int ch;                   // K slices per TMEM chunk
  float* C;                 // output: C + z * split_stride, column-major, ldc
  int64_t ldc;
  int64_t split_stride;
  const unsigned* bmax;     // raw B: per-column bound on |B| (float bits), column 0 = B's first column
  double* nrm2;             // raw B, optional: += sum of B[r, c]^2 over this CTA's rows (FP64 atomics)
  float out_scale;          // uniform factor of every output (1 / (s_A s_B), s_B = 1 for raw B)
  int* status;
};

// Threads of k_tc_gemm16: DW = 1 drains each M tile's 128 columns with one
// warpgroup (whose first four warps also split raw B); DW = 2 drains them with
// two warpgroups of 64 columns each, beside four warps that only split.
__host__ __device__ constexpr int g16_threads(int MT, int DW) { return DW == 1 ? 64 + 128 * MT : 192 + 128 * MT * DW; }

// W = A^T B, see the file comment.  Warps: 0 TMA producer, 1 TMEM owner and
// MMA issuer; DW = 1: 2 .. 2 + 4 MT - 1 drain the accumulators (warps 2-5
// also split raw B slices); DW = 2: 2-5 split raw B, 6 .. 6 + 8 MT - 1 drain
// (64 accumulator columns each, so every thread fits in the smaller register
// share of the larger CTA).
template <int MT, bool BRAW, int STAGES, int DW>
__global__ void __launch_bounds__(g16_threads(MT, DW), 1) __maxnreg__(DW == 2 ? 88 : (MT == 2 ? 200 : 255))
    k_tc_gemm16(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, G16Args args) {
  // Operand ring (STAGES deep): A's [mt][h, l] tiles, then B's FP16 h, l
  // tiles, or for raw B its FP32 slice.  Raw B is split into a separate
  // two-slot ring of FP16 h, l tiles, so the deep ring holds only what TMA
  // loads (more slices in flight for the same shared memory).
  constexpr uint32_t A_OFF = 0;
  constexpr uint32_t B_OFF = MT * 2 * kT16;            // B h, B l (pre-split B)
  constexpr uint32_t R_OFF = MT * 2 * kT16;            // raw B (BRAW)
  constexpr uint32_t STAGE_BYTES = MT * 2 * kT16 + (BRAW ? kTRaw : 2 * kT16);
  constexpr uint32_t TX_BYTES = STAGE_BYTES;
  constexpr uint32_t HL_BYTES = BRAW ? 2 * (2 * kT16) : 0;
  constexpr uint32_t TMEM_COLS = 2 * MT * kBN;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* hl = smem + STAGES * STAGE_BYTES;     // [2][h, l] split raw B slices
  uint64_t* full = (uint64_t*)(hl + HL_BYTES);
  uint64_t* conv = full + STAGES;
  uint64_t* empty = conv + STAGES;
  uint64_t* tfull = empty + STAGES;  // [2] a chunk's MMAs are done in TMEM buffer b
  uint64_t* tempty = tfull + 2;      // [2] every drain warp has read buffer b
  uint64_t* hlempty = tempty + 2;    // [2] the MMAs have read split slot h
  uint32_t* tmem_slot = (uint32_t*)(hlempty + 2);
  float* colinv = (float*)(tmem_slot + 4);  // [kBN] 1 / (per-column scale of raw B)

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * (kBM * MT), n0 = (int64_t)blockIdx.y * kBN;
  const int64_t kbeg = (int64_t)blockIdx.z * args.k_chunk;
  int64_t kend = kbeg + args.k_chunk;
  if (kend > args.K) kend = args.K;
  const int nk = kend > kbeg ? (int)((kend - kbeg + kBK - 1) / kBK) : 0;
  const int CH = args.ch > 0 ? args.ch : 1;
  const int nch = (nk + CH - 1) / CH;

  // converter thread t (warps 2-5) owns B tile row t = column n0 + t
  float bsc = 1.f, inv = 1.f;
  if (threadIdx.x >= 64 && threadIdx.x < 192) {
    const int t = threadIdx.x - 64;
    if (BRAW && n0 + t < args.N) {
      const float amax = __uint_as_float(__ldg(args.bmax + n0 + t));
      if (amax > 0.f && isfinite(amax)) {
        int e;
        frexpf(amax, &e);  // amax < 2^e
        int k = 14 - e;
        k = k < -126 ? -126 : (k > 126 ? 126 : k);
        bsc = ldexpf(1.f, k);
        inv = ldexpf(1.f, -k);
      }
    }
    colinv[t] = inv;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 4);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4 * MT * DW);
      mbar_init(&hlempty[b], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      for (int kt = 0; kt < nk && ok; ++kt) {
        const int s = kt % STAGES, u = kt / STAGES;
        if (u > 0 && !mbar_wait(&empty[s], (uint32_t)((u - 1) & 1), args.status)) { ok = false; break; }
        unsigned char* st = smem + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], TX_BYTES);
        const int x = (int)(kbeg + (int64_t)kt * kBK);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          tma_load_2d(st + A_OFF + (2 * mt) * kT16, &tmAh, x, (int)(m0 + mt * kBM), &full[s]);
          tma_load_2d(st + A_OFF + (2 * mt + 1) * kT16, &tmAl, x, (int)(m0 + mt * kBM), &full[s]);
        }
        if (BRAW) {
          tma_load_2d(st + R_OFF, &tmBh, x, (int)n0, &full[s]);
        } else {
          tma_load_2d(st + B_OFF, &tmBh, x, (int)n0, &full[s]);
          tma_load_2d(st + B_OFF + kT16, &tmBl, x, (int)n0, &full[s]);
        }
        ++issued;
      }
      if (!ok) {
        // Error exit: let the copies already issued land before the CTA ends.
        for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
          mbar_wait(&full[kt % STAGES], (uint32_t)((kt / STAGES) & 1), args.status, false);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(kBN);
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % STAGES, u = kt / STAGES;
        const int c = kt / CH, b = c & 1;
        const bool first = kt % CH == 0;
        // buffer b must have been read out for chunk c - 2
        if (first && c >= 2 && !mbar_wait(&tempty[b], (uint32_t)(((c >> 1) - 1) & 1), args.status)) break;
        if (!mbar_wait(BRAW ? &conv[s] : &full[s], (uint32_t)(u & 1), args.status)) break;
        tc_fence_after();
        unsigned char* st = smem + s * STAGE_BYTES;
        unsigned char* bt = BRAW ? hl + (kt & 1) * (2 * kT16) : st + B_OFF;
        const uint64_t dbh = sdesc_sw64(bt), dbl = sdesc_sw64(bt + kT16);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 2);  // 16 FP16 = 32 bytes = 2 x 16 B
#pragma unroll
          for (int mt = 0; mt < MT; ++mt) {
            const uint64_t dah = sdesc_sw64(st + A_OFF + (2 * mt) * kT16);
            const uint64_t dal = sdesc_sw64(st + A_OFF + (2 * mt + 1) * kT16);
            const uint32_t d = tmem + (uint32_t)((b * MT + mt) * kBN);
            mma_f16_ss(d, dah + adv, dbh + adv, idesc, (!first || kk > 0) ? 1u : 0u);
            mma_f16_ss(d, dal + adv, dbh + adv, idesc, 1u);
            mma_f16_ss(d, dah + adv, dbl + adv, idesc, 1u);
          }
        }
        mma_commit(&empty[s]);
        if (BRAW) mma_commit(&hlempty[kt & 1]);
        if (kt % CH == CH - 1 || kt == nk - 1) mma_commit(&tfull[b]);
      }
    }
  } else {
    // DW = 1: warps 2 .. 2 + 4 MT - 1; DW = 2: converters 2-5, drains 6 ..
    constexpr int D0 = DW == 1 ? 2 : 6;  // first drain warp
    constexpr int NC = kBN / DW;         // accumulator columns per drain thread
    // Split raw B slice kt into FP16 h, l parts (warps 2-5, thread t owns
    // column n0 + t); false when a wait gave up.
    auto convert = [&](int kt, float& ssq) -> bool {
      const int t = (warp - 2) * 32 + lane;
      const int sw_in = t & 7, sw_out = (t >> 1) & 3;
      const int s = kt % STAGES, u = kt / STAGES;
      if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (uint32_t)(u & 1), args.status))) return false;
      // split slot kt & 1 must have been read by slice kt - 2's MMAs
      if (kt >= 2 &&
          !__all_sync(0xffffffffu, mbar_wait(&hlempty[kt & 1], (uint32_t)(((kt >> 1) - 1) & 1), args.status)))
        return false;
      unsigned char* st = smem + s * STAGE_BYTES;
      const unsigned char* raw = st + R_OFF + t * 128;
      unsigned char* bh = hl + (kt & 1) * (2 * kT16) + t * 64;
      unsigned char* bl = bh + kT16;
      // one 16-byte output chunk at a time: few live registers beside the
      // accumulators that DW = 1 converter threads also hold
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        const float4 x0 = *(const float4*)(raw + (((2 * q) ^ sw_in) << 4));
        const float4 x1 = *(const float4*)(raw + (((2 * q + 1) ^ sw_in) << 4));
        __half h[8], l[8];
        float xs[8];
        xs[0] = split16(x0.x, bsc, h[0], l[0]);
        xs[1] = split16(x0.y, bsc, h[1], l[1]);
        xs[2] = split16(x0.z, bsc, h[2], l[2]);
        xs[3] = split16(x0.w, bsc, h[3], l[3]);
        xs[4] = split16(x1.x, bsc, h[4], l[4]);
        xs[5] = split16(x1.y, bsc, h[5], l[5]);
        xs[6] = split16(x1.z, bsc, h[6], l[6]);
        xs[7] = split16(x1.w, bsc, h[7], l[7]);
        if (args.nrm2) {
#pragma unroll
          for (int v = 0; v < 8; ++v) ssq = fmaf(xs[v], xs[v], ssq);
        }
        const int o = (q ^ sw_out) << 4;
        *(uint4*)(bh + o) = make_uint4(pack2(h[0], h[1]), pack2(h[2], h[3]), pack2(h[4], h[5]), pack2(h[6], h[7]));
        *(uint4*)(bl + o) = make_uint4(pack2(l[0], l[1]), pack2(l[2], l[3]), pack2(l[4], l[5]), pack2(l[6], l[7]));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[s]);
      return true;
    };
    // the sum of squares of column n0 + t, back at its original scale
    auto add_nrm2 = [&](float ssq) {
      const int t = (warp - 2) * 32 + lane;
      if (args.nrm2 && ssq > 0.f && n0 + t < args.N)
        atomicAdd(args.nrm2 + n0 + t, (double)ssq * (double)inv * (double)inv);
    };
    if (DW == 2 && BRAW && warp < 6) {
      float ssq = 0.f;
      bool ok = true;
      for (int kt = 0; kt < nk && ok; ++kt) ok = convert(kt, ssq);
      if (ok) add_nrm2(ssq);
    } else {
      const int g = (warp - D0) >> 2;
      const int mt = g / DW, c0 = (g % DW) * NC;
      const int lg = warp & 3;  // TMEM lanes 32 lg .. +31 = tile rows
      float acc[NC];
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[j] = 0.f;
      int next = 0;  // next chunk to read out
      bool ok = true;
      auto drain = [&](int c) -> bool {
        const int b = c & 1;
        // warp-uniform decision: the TMEM loads below are .sync.aligned
        if (!__all_sync(0xffffffffu, mbar_wait(&tfull[b], (uint32_t)((c >> 1) & 1), args.status))) return false;
        tc_fence_after();
        constexpr int LW = DW == 1 ? 16 : 8;  // columns per TMEM load
#pragma unroll
        for (int cc = 0; cc < NC; cc += LW) {
          float v[LW];
          const uint32_t ta = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)((b * MT + mt) * kBN + c0 + cc);
          if (LW == 16) tmem_ld16(ta, v); else tmem_ld8(ta, v);
#pragma unroll
          for (int j = 0; j < LW; ++j) acc[cc + j] += v[j];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
        return true;
      };
      if (DW == 1 && BRAW && warp < 6) {
        float ssq = 0.f;
        for (int kt = 0; kt < nk && ok; ++kt) {
          ok = convert(kt, ssq);
          // the chunk before the one this slice completes is long done
          if (ok && kt % CH == CH - 1)
            while (next < kt / CH && ok) ok = drain(next++);
        }
        if (ok) add_nrm2(ssq);
      }
      while (next < nch && ok) ok = drain(next++);
      if (ok) {
        const int64_t row = m0 + mt * kBM + lg * 32 + lane;
        if (row < args.M) {
          const int nv = (int)(args.N - n0 < kBN ? args.N - n0 : kBN) - c0;
          float* p = args.C + (int64_t)blockIdx.z * args.split_stride + row + (n0 + c0) * args.ldc;
#pragma unroll
          for (int j = 0; j < NC; ++j) {
            if (j < nv) *p = acc[j] * args.out_scale * colinv[c0 + j];
            p += args.ldc;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

struct U16Args {
  int64_t M, N, K;
  float* C;
  int64_t ldc;
  int64_t mtiles, ntiles;
  const float* colinv;   // per column of B: 1 / (s_A s_B[c]), readable up to a multiple of 128 columns
  int* status;
};

// Output tile t of the persistent update -> first row m0 and column n0, in
// bands of G = gridDim.x row tiles (each CTA keeps one row tile, so V and W'
// tiles are read from DRAM once per band; see tc_gemm.cu).
__device__ __forceinline__ void tile_of(int64_t t, int64_t mtiles, int64_t ntiles, int64_t G, int64_t& m0,
                                        int64_t& n0) {
  // 32-bit index arithmetic (the host keeps the tile count below 2^31)
  const uint32_t tt = (uint32_t)t, g = (uint32_t)G, nt = (uint32_t)ntiles, mt = (uint32_t)mtiles;
  const uint32_t band = tt / (g * nt), local = tt - band * g * nt;
  const uint32_t rows = mt - band * g < g ? mt - band * g : g;
  m0 = (int64_t)(band * g + local % rows) * kBM;
  n0 = (int64_t)(local / rows) * kBN;
}

// C -= A^T B on pre-split operands, see the file comment.  Warps: 0 TMA
// producer, 1 MMA issuer, 4-11 epilogue (row lg*32 + lane, 64 columns each).
template <int STAGES>
__global__ void __launch_bounds__(kUpdThreads, 1)
    k_tc_update16(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                  const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, U16Args args) {
  constexpr uint32_t STAGE_BYTES = 4 * kUTile;  // A h, B h, A l, B l
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntile = args.mtiles * args.ntiles;
  const int nk = (int)((args.K + kUK - 1) / kUK);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 8);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(256u)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int64_t g = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
        int64_t m0l, n0l;
        tile_of(t, args.mtiles, args.ntiles, gridDim.x, m0l, n0l);
        const int m0 = (int)m0l, n0 = (int)n0l;
        for (int ks = 0; ks < nk; ++ks, ++g) {
          const int s = (int)(g % STAGES);
          const int64_t u = g / STAGES;
          if (u > 0 && !mbar_wait(&empty[s], (uint32_t)((u - 1) & 1), args.status)) { ok = false; break; }
          unsigned char* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          const int x = ks * kUK;
          tma_load_2d(st, &tmAh, x, m0, &full[s]);
          tma_load_2d(st + kUTile, &tmBh, x, n0, &full[s]);
          tma_load_2d(st + 2 * kUTile, &tmAl, x, m0, &full[s]);
          tma_load_2d(st + 3 * kUTile, &tmBl, x, n0, &full[s]);
        }
      }
      if (!ok) {
        for (int64_t q = (g > STAGES ? g - STAGES : 0); q < g; ++q)
          mbar_wait(&full[q % STAGES], (uint32_t)((q / STAGES) & 1), args.status, false);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(kBN);
      int64_t g = 0;
      int it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x, ++it) {
        const int acc = it & 1, ua = it >> 1;
        if (ua > 0 && !mbar_wait(&tempty[acc], (uint32_t)((ua - 1) & 1), args.status)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * kBN);
        for (int ks = 0; ks < nk; ++ks, ++g) {
          const int s = (int)(g % STAGES);
          const int64_t u = g / STAGES;
          if (!mbar_wait(&full[s], (uint32_t)(u & 1), args.status)) { ok = false; break; }
          tc_fence_after();
          unsigned char* st = smem + s * STAGE_BYTES;
          const uint64_t dah = sdesc_sw128(st), dbh = sdesc_sw128(st + kUTile);
          const uint64_t dal = sdesc_sw128(st + 2 * kUTile), dbl = sdesc_sw128(st + 3 * kUTile);
#pragma unroll
          for (int kk = 0; kk < kUK / 16; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 2);
            mma_f16_ss(d, dah + adv, dbh + adv, idesc, (ks > 0 || kk > 0) ? 1u : 0u);
            mma_f16_ss(d, dal + adv, dbh + adv, idesc, 1u);
            mma_f16_ss(d, dah + adv, dbl + adv, idesc, 1u);
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&tfull[acc]);
      }
    }
  } else if (warp >= 4) {
    const int lg = warp & 3, half = (warp - 4) >> 2;
    const int et = threadIdx.x - 128;
    float* cbuf = (float*)(smem + STAGES * STAGE_BYTES + 256);
    const int64_t ldc = args.ldc;
    auto prefetch = [&](int64_t t) {
      int64_t m0, n0;
      tile_of(t, args.mtiles, args.ntiles, gridDim.x, m0, n0);
      const int64_t row = m0 + lg * 32 + lane, c0 = n0 + half * 64;
      const int nv = row < args.M ? (int)(args.N - c0 < 64 ? args.N - c0 : 64) : 0;
      const float* p = args.C + row + c0 * ldc;
#pragma unroll 16
      for (int j = 0; j < 64; ++j) {
        cp_async_f32(cbuf + j * 256 + et, j < nv ? p : args.C, j < nv);
        p += ldc;
      }
      cp_async_commit();
    };
    if ((int64_t)blockIdx.x < ntile) prefetch(blockIdx.x);
    int it = 0;
    for (int64_t t = blockIdx.x; t < ntile; t += gridDim.x, ++it) {
      const int acc = it & 1, ua = it >> 1;
      int64_t m0, n0;
      tile_of(t, args.mtiles, args.ntiles, gridDim.x, m0, n0);
      const int64_t row = m0 + lg * 32 + lane;
      const int64_t c0 = n0 + half * 64;
      const bool rok = row < args.M;
      float c[64];
      cp_async_wait_all();
#pragma unroll
      for (int j = 0; j < 64; ++j) c[j] = cbuf[j * 256 + et];
      if (t + gridDim.x < ntile) prefetch(t + gridDim.x);
      if (!__all_sync(0xffffffffu, mbar_wait(&tfull[acc], (uint32_t)(ua & 1), args.status))) {
        cp_async_wait_all();
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(acc * kBN + half * 64 + q * 16), v);
        // the 16 columns' inverse scales (colinv is padded to whole tiles)
#pragma unroll
        for (int i = 0; i < 16; i += 4) {
          const float4 w4 = __ldg((const float4*)(args.colinv + c0 + q * 16 + i));
          c[q * 16 + i] -= v[i] * w4.x;
          c[q * 16 + i + 1] -= v[i + 1] * w4.y;
          c[q * 16 + i + 2] -= v[i + 2] * w4.z;
          c[q * 16 + i + 3] -= v[i + 3] * w4.w;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
      if (rok) {
        const int nv = (int)(args.N - c0 < 64 ? args.N - c0 : 64);
        float* p = args.C + row + c0 * ldc;
#pragma unroll
        for (int j = 0; j < 64; ++j) {
          if (j < nv) *p = c[j];
          p += ldc;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
  }
}

// ---- small helpers -----------------------------------------------------------

// bound[c] = bits of a float >= ||X[0:rows, c]||_2 (FP64 sums of squares per
// warp and row range of 8192, added atomically in FP64 into acc).
__global__ void __launch_bounds__(256) k_colnorm2(const float* __restrict__ X, int64_t ldx, int64_t rows,
                                                  int64_t cols, double* __restrict__ acc) {
  const int64_t c = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= cols) return;
  const int64_t r0 = (int64_t)blockIdx.y * 8192;
  int64_t r1 = r0 + 8192;
  if (r1 > rows) r1 = rows;
  const float* x = X + c * ldx;
  double s2 = 0.0;
  for (int64_t r = r0 + lane; r < r1; r += 32) {
    const double v = (double)__ldcs(x + r);
    s2 = fma(v, v, s2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if (lane == 0 && s2 > 0.0) atomicAdd(acc + c, s2);
}

// bound[c] = bits of (float) sqrt(acc[c]) rounded up, times (1 + 2^-10) for
// the rounding of the FP32 updates that follow.
__global__ void __launch_bounds__(256) k_norm_bound(const double* __restrict__ acc, int64_t cols,
                                                    unsigned* __restrict__ bound) {
  const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (c >= cols) return;
  const double nrm = sqrt(acc[c]) * (1.0 + 1.0 / 1024.0);
  bound[c] = __float_as_uint(__double2float_ru(nrm));
}

// H + L = X * s (FP16 parts, same K x cols layout, ldo) with s = 2^e: e fixed
// (exp_fixed) when cmax is NULL, else per column from cmax (a bound on the
// column's magnitudes, below 2^14 after scaling); colinv[c] = 2^-(e + extra_exp).
__global__ void __launch_bounds__(256) k_split16_cols(const float* __restrict__ X, int64_t ldx, int64_t K,
                                                      int64_t cols, const unsigned* __restrict__ cmax, int exp_fixed,
                                                      int extra_exp, __half* __restrict__ H, __half* __restrict__ L,
                                                      int64_t ldo, float* __restrict__ colinv) {
  const int64_t c = blockIdx.y;
  if (c >= cols) return;
  int e = exp_fixed;
  if (cmax) {
    e = 0;
    const float amax = __uint_as_float(cmax[c]);
    if (amax > 0.f && isfinite(amax)) {
      int ex;
      frexpf(amax, &ex);
      e = 14 - ex;
      e = e < -126 ? -126 : (e > 126 ? 126 : e);
    }
  }
  const float s = ldexpf(1.f, e);
  if (colinv && blockIdx.x == 0 && threadIdx.x == 0) colinv[c] = ldexpf(1.f, -(e + extra_exp));
  for (int64_t r = (int64_t)blockIdx.x * 256 + threadIdx.x; r < K; r += (int64_t)gridDim.x * 256) {
    __half h, l;
    split16(X[r + c * ldx], s, h, l);
    H[r + c * ldo] = h;
    L[r + c * ldo] = l;
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn16() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// 2-D tensor: d0 contiguous elements per column, d1 columns, column stride ld
// elements of esize bytes; boxes of box0 x box1.
bool make_map16(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esize, uint64_t d0, uint64_t d1,
                uint64_t ld, uint32_t box0, uint32_t box1, CUtensorMapSwizzle sw) {
  EncodeTiledFn fn = encode_fn16();
  if (!fn) return false;
  cuuint64_t dims[2] = {d0, d1};
  cuuint64_t strides[1] = {ld * (uint64_t)esize};
  cuuint32_t box[2] = {box0, box1};
  cuuint32_t es[2] = {1, 1};
  return fn(m, dt, 2, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MT, bool BRAW, int STAGES, int DW = 1>
ct_status launch_g16(const CUtensorMap* maps, const G16Args& a, int splits, cudaStream_t s) {
  constexpr size_t STAGE_BYTES = (size_t)MT * 2 * kT16 + (BRAW ? kTRaw : 2 * kT16);
  constexpr size_t HL_BYTES = BRAW ? 4 * kT16 : 0;
  const size_t smem = STAGES * STAGE_BYTES + HL_BYTES + 1024 + 256 + kBN * sizeof(float);
  static bool attr_done = false;
  if (!attr_done) {
    CT_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm16<MT, BRAW, STAGES, DW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    attr_done = true;
  }
  const dim3 grid((unsigned)((a.M + kBM * MT - 1) / (kBM * MT)), (unsigned)((a.N + kBN - 1) / kBN),
                  (unsigned)splits);
  k_tc_gemm16<MT, BRAW, STAGES, DW><<<grid, g16_threads(MT, DW), smem, s>>>(maps[0], maps[1], maps[2], maps[3], a);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

}  // namespace

// W (M x N) = A^T B, see the file comment.  Ah/Al: K x M FP16 parts (ld lda,
// a multiple of 8), scale 1/out_scale folded in by the caller; B either FP32
// (Bl == NULL, Bh = the FP32 matrix, ld ldb multiple of 4; bmax bounds on its
// columns' magnitudes; nrm2, when given, receives += each column's sum of
// squares over K, added in FP64 by every split) or FP16 parts (Bh, Bl, ld ldb
// multiple of 8).
// Split z of `splits` (over K, chunks rounded to 32 rows) writes
// C + z * split_stride.  Returns the number of splits made in *made.
ct_status tc_gemm16(const __half* Ah, const __half* Al, int64_t lda, const void* Bh, const __half* Bl, int64_t ldb,
                    const unsigned* bmax, double* nrm2, int64_t M, int64_t N, int64_t K, float out_scale, float* C,
                    int64_t ldc, int64_t split_stride, int splits, int* status, cudaStream_t s, int* made) {
  const bool braw = Bl == nullptr;
  if (made) *made = 0;
  if (M <= 0 || N <= 0) return CT_OK;
  if (!Ah || !Al || !Bh || !C || K < 0 || lda < K || ldb < K || ldc < M || (braw && !bmax)) return CT_ERR_INVALID;
  if (((uintptr_t)Ah & 15) || ((uintptr_t)Al & 15) || ((uintptr_t)Bh & 15) || ((uintptr_t)Bl & 15) || (lda & 7) ||
      (braw ? (ldb & 3) : (ldb & 7)))
    return CT_ERR_INVALID;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return CT_ERR_INVALID;
  if (splits < 1) splits = 1;
  int64_t chunk = (K + splits - 1) / splits;
  chunk = (chunk + kBK - 1) / kBK * kBK;
  if (chunk < kBK) chunk = kBK;
  splits = (int)((K + chunk - 1) / chunk);
  if (splits < 1) splits = 1;
  if (splits > 1 && split_stride < ldc * N) return CT_ERR_INVALID;
  const uint64_t kd = K > 0 ? (uint64_t)K : 1;
  CUtensorMap maps[4];
  if (!make_map16(&maps[0], Ah, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, kd, (uint64_t)M, (uint64_t)lda, kBK, kBM,
                  CU_TENSOR_MAP_SWIZZLE_64B) ||
      !make_map16(&maps[1], Al, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, kd, (uint64_t)M, (uint64_t)lda, kBK, kBM,
                  CU_TENSOR_MAP_SWIZZLE_64B))
    return CT_ERR_CUDA;
  if (braw) {
    if (!make_map16(&maps[2], Bh, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, kd, (uint64_t)N, (uint64_t)ldb, kBK, kBN,
                    CU_TENSOR_MAP_SWIZZLE_128B))
      return CT_ERR_CUDA;
    maps[3] = maps[2];
  } else if (!make_map16(&maps[2], Bh, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, kd, (uint64_t)N, (uint64_t)ldb, kBK, kBN,
                         CU_TENSOR_MAP_SWIZZLE_64B) ||
             !make_map16(&maps[3], Bl, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, kd, (uint64_t)N, (uint64_t)ldb, kBK, kBN,
                         CU_TENSOR_MAP_SWIZZLE_64B)) {
    return CT_ERR_CUDA;
  }
  G16Args a;
  a.M = M;
  a.N = N;
  a.K = K;
  a.k_chunk = chunk;
  a.ch = kChunkSlices;
  a.C = C;
  a.ldc = ldc;
  a.split_stride = split_stride;
  a.bmax = bmax;
  a.nrm2 = braw ? nrm2 : nullptr;
  a.out_scale = out_scale;
  a.status = status;
  if (made) *made = splits;
  LaunchScope ls(K_TC_GEMM, s, 2.0 * M * N * K, 4.0 * (double)K * (M + N) + 4.0 * M * N * splits);
  // Two M tiles per CTA when M > 128: C is read and split once for all 256
  // reflectors (one M tile per CTA was measured 1.6x slower on a 50,000 x
  // 12,544 x 256 product).  With raw B, four warps only split and two
  // warpgroups per M tile drain 64 columns each (DW = 2): the V^T C class of
  // the 256 x 256 system's factorization fell from 1.81 s to 1.48 s against
  // DW = 1, whose split warps also hold 128 accumulators and spill.
  const bool two = M > kBM;
  if (braw) return two ? launch_g16<2, true, 4, 2>(maps, a, splits, s) : launch_g16<1, true, 6>(maps, a, splits, s);
  return two ? launch_g16<2, false, 4>(maps, a, splits, s) : launch_g16<1, false, 6>(maps, a, splits, s);
}

int tc_gemm16_m_ctas(int64_t M) {
  const int per = M > kBM ? 2 * kBM : kBM;
  return (int)((M + per - 1) / per);
}

// C (M x N) -= A^T B on pre-split operands (Ah/Al: K x M, Bh/Bl: K x N, FP16
// column-major, ld multiples of 8, K <= 256) with colinv[c] = 1 / (s_A s_B[c])
// (16-byte aligned and readable up to N rounded up to 128 entries).
ct_status tc_update16(const __half* Ah, const __half* Al, int64_t lda, const __half* Bh, const __half* Bl, int64_t ldb,
                      const float* colinv, int64_t M, int64_t N, int64_t K, float* C, int64_t ldc, int sms, int* status,
                      cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return CT_OK;
  if (!Ah || !Al || !Bh || !Bl || !C || !colinv || lda < K || ldb < K || ldc < M) return CT_ERR_INVALID;
  if (((uintptr_t)Ah & 15) || ((uintptr_t)Al & 15) || ((uintptr_t)Bh & 15) || ((uintptr_t)Bl & 15) || (lda & 7) ||
      (ldb & 7))
    return CT_ERR_INVALID;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return CT_ERR_INVALID;
  CUtensorMap maps[4];
  if (!make_map16(&maps[0], Ah, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (uint64_t)K, (uint64_t)M, (uint64_t)lda, kUK, kBM,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map16(&maps[1], Al, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (uint64_t)K, (uint64_t)M, (uint64_t)lda, kUK, kBM,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map16(&maps[2], Bh, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, kUK, kBN,
                  CU_TENSOR_MAP_SWIZZLE_128B) ||
      !make_map16(&maps[3], Bl, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, kUK, kBN,
                  CU_TENSOR_MAP_SWIZZLE_128B))
    return CT_ERR_CUDA;
  U16Args a;
  a.M = M;
  a.N = N;
  a.K = K;
  a.C = C;
  a.ldc = ldc;
  a.mtiles = (M + kBM - 1) / kBM;
  a.ntiles = (N + kBN - 1) / kBN;
  if (a.mtiles * a.ntiles + sms > INT32_MAX) return CT_ERR_INVALID;  // 32-bit tile indices
  a.colinv = colinv;
  a.status = status;
  constexpr int STAGES = kUStages;
  const size_t smem = STAGES * (size_t)(4 * kUTile) + 1024 + 256 + kUpdCbufBytes;
  static bool attr_done = false;
  if (!attr_done) {
    CT_CUDA_TRY(cudaFuncSetAttribute(k_tc_update16<STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_done = true;
  }
  const int64_t tiles = a.mtiles * a.ntiles;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
  LaunchScope ls(K_TC_UPDATE, s, 2.0 * M * N * K, 4.0 * (double)K * (M + N) + 8.0 * M * N);
  k_tc_update16<STAGES><<<grid, kUpdThreads, smem, s>>>(maps[0], maps[1], maps[2], maps[3], a);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

// bound[c] = bits of a float above ||X[0:rows, c]||_2, a bound on every
// |X[r, c]| that the orthogonal updates of later outer blocks keep (they
// preserve the 2-norm of each column's rows from J down, so the norm over
// fewer rows can only shrink).  acc: cols doubles of scratch.
ct_status launch_norm_bound(const double* nrm2, int64_t cols, unsigned* bound, cudaStream_t s) {
  if (cols <= 0) return CT_OK;
  LaunchScope ls(K_COPY, s, 0.0, 12.0 * (double)cols);
  k_norm_bound<<<(unsigned)((cols + 255) / 256), 256, 0, s>>>(nrm2, cols, bound);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

ct_status launch_colnorm_bound(const float* X, int64_t ldx, int64_t rows, int64_t cols, double* acc, unsigned* bound,
                               cudaStream_t s) {
  if (cols <= 0) return CT_OK;
  CT_CUDA_TRY(cudaMemsetAsync(acc, 0, (size_t)cols * sizeof(double), s));
  const int64_t ry = rows > 0 ? (rows + 8191) / 8192 : 0;
  if (ry > 65535) return CT_ERR_INVALID;
  LaunchScope ls(K_COPY, s, 2.0 * (double)rows * cols, 4.0 * (double)rows * cols);
  if (ry > 0) {
    k_colnorm2<<<dim3((unsigned)((cols + 7) / 8), (unsigned)ry), 256, 0, s>>>(X, ldx, rows, cols, acc);
    CT_LAUNCH_CHECK();
  }
  k_norm_bound<<<(unsigned)((cols + 255) / 256), 256, 0, s>>>(acc, cols, bound);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

// FP16 parts of X (K x cols FP32, ld ldx) into H/L (ld ldo): scale 2^exp_fixed,
// or per column from cmax when given; colinv[c] = 2^-(e_c + extra_exp).
ct_status launch_split16(const float* X, int64_t ldx, int64_t K, int64_t cols, const unsigned* cmax, int exp_fixed,
                         int extra_exp, __half* H, __half* L, int64_t ldo, float* colinv, cudaStream_t s) {
  if (K <= 0 || cols <= 0) return CT_OK;
  if (cols > 65535) return CT_ERR_INVALID;
  int gx = (int)((K + 255) / 256);
  if (gx > 64) gx = 64;
  LaunchScope ls(K_COPY, s, 0.0, 8.0 * (double)K * cols);
  k_split16_cols<<<dim3((unsigned)gx, (unsigned)cols), 256, 0, s>>>(X, ldx, K, cols, cmax, exp_fixed, extra_exp, H,
                                                                     L, ldo, colinv);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

}  // namespace ctqr
