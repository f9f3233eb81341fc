// tc_gemm.cu -- tensor-core (tcgen05, TF32) GEMM for the trailing update.
//
//   C (M x N)  =  A^T B        (mode 0: store; split z writes C + z*split_stride)
//   C (M x N) -=  A^T B        (mode 1)
// with A stored K x M and B stored K x N, both column-major FP32 (so both
// operands are K-major, the canonical tcgen05 layout), C column-major FP32.
// This one "TN" form covers both contractions of the block-reflector update
// C <- C - V (T^T (V^T C)) (the paper's Apply_left_Qt_of_dense_QR task):
// V^T C uses A = V (column-major) and B = C; the update V W uses A = V stored
// row-major (K = reflectors contiguous) and B = W.
//
// Structure (one 128 x BN output tile per CTA, optional split-K over z):
//   warp 0 (one lane)  TMA producer: 128B-swizzled 32-float K slices of A and
//                      B into a STAGES-deep shared-memory ring, mbarrier
//                      expect_tx completion;
//   warp 1 (one lane)  allocates TMEM and issues tcgen05.mma.kind::tf32
//                      (M = 128, N = BN, K = 8 each, 4 per slice), committing
//                      each stage back to the producer; the K range is cut
//                      into chunks of CH slices accumulated alternately in two
//                      TMEM buffers (see below);
//   warps 2-5          split3: turn each landed slice x into a TF32-exact high
//                      part hi = trunc_tf32(x) (in place) and a low part
//                      lo = x - hi, so the three products hi*hi + hi*lo + lo*hi
//                      recover FP32-level accuracy (error-compensated TF32);
//                      as each chunk completes they add its TMEM buffer into
//                      an FP32 register accumulator (tcgen05.ld, one row per
//                      thread) and release the buffer; at the end they apply
//                      the epilogue (column-major stores).
// Why chunks: the tensor cores' FP32 accumulation rounds each MMA's sum
// towards zero, so one accumulator over a long K (the V^T C product runs
// over all rows of the trailing matrix, up to 135,232) drifts by about
// K/8 * 3 truncations of its running value: relative errors near 1e-2 at
// that height, which wrecked the preconditioner of the 256 x 256 system.
// Restarting the TMEM accumulation every CH slices and summing the chunks on
// the CUDA cores (round to nearest) bounds the drift by the chunk length.
// Every wait is bounded (CT_ERR_TIMEOUT in the status word, then an orderly
// exit that still waits for issued copies and MMAs and frees TMEM).
#include <cuda.h>

#include "internal.cuh"
#include "tcgen05.cuh"

namespace ctqr {
namespace {

using namespace tc;

constexpr int kBM = 128;
constexpr int kBK = 32;  // floats per K slice = one 128-byte swizzle row
constexpr int kThreads = 192;
// K slices (of kBK rows) per TMEM accumulation chunk: 256 rows, about 96
// truncating accumulations of 3xTF32 MMAs per chunk.
constexpr int kAccChunkSlices = 8;

struct TcArgs {
  int64_t M, N, K;
  int64_t k_chunk;   // K rows per split (blockIdx.z)
  int ch;            // K slices per TMEM accumulation chunk
  float* C;
  int64_t ldc;
  int64_t split_stride;
  int mode;
  int* status;
};

__device__ __forceinline__ float tf32_trunc(float x) {
  return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

template <int BN, int STAGES, bool SPLIT3>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm_tn(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs args) {
  constexpr uint32_t A_BYTES = kBM * kBK * 4;
  constexpr uint32_t B_BYTES = BN * kBK * 4;
  constexpr uint32_t STAGE_BYTES = (A_BYTES + B_BYTES) * (SPLIT3 ? 2 : 1);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* conv = full + STAGES;
  uint64_t* empty = conv + STAGES;
  uint64_t* tfull = empty + STAGES;   // [2] a chunk's MMAs are done in TMEM buffer b
  uint64_t* tempty = tfull + 2;       // [2] the epilogue warps have read buffer b
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * kBM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * args.k_chunk;
  int64_t kend = kbeg + args.k_chunk;
  if (kend > args.K) kend = args.K;
  const int nk = kend > kbeg ? (int)((kend - kbeg + kBK - 1) / kBK) : 0;
  const int CH = args.ch > 0 ? args.ch : 1;
  const int nch = (nk + CH - 1) / CH;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 4);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)(2 * BN))
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
        mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
        const int x = (int)(kbeg + (int64_t)kt * kBK);
        tma_load_2d(st, &tmA, x, (int)m0, &full[s]);
        tma_load_2d(st + A_BYTES, &tmB, x, (int)n0, &full[s]);
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
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                             ((uint32_t)(kBM >> 4) << 24);
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % STAGES, u = kt / STAGES;
        const int c = kt / CH, b = c & 1;
        const bool first = kt % CH == 0;
        // buffer b must have been read out for chunk c - 2
        if (first && c >= 2 && !mbar_wait(&tempty[b], (uint32_t)(((c >> 1) - 1) & 1), args.status)) break;
        if (!mbar_wait(SPLIT3 ? &conv[s] : &full[s], (uint32_t)(u & 1), args.status)) break;
        tc_fence_after();
        unsigned char* st = smem + s * STAGE_BYTES;
        const uint64_t da = sdesc_sw128(st), db = sdesc_sw128(st + A_BYTES);
        const uint32_t d = tmem + (uint32_t)(b * BN);
#pragma unroll
        for (int kk = 0; kk < kBK / 8; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 2);  // 8 floats = 32 bytes = 2 x 16 B
          mma_tf32(d, da + adv, db + adv, idesc, (!first || kk > 0) ? 1u : 0u);
          if (SPLIT3) {
            const uint64_t dal = sdesc_sw128(st + A_BYTES + B_BYTES);
            const uint64_t dbl = sdesc_sw128(st + 2 * A_BYTES + B_BYTES);
            mma_tf32(d, dal + adv, db + adv, idesc, 1u);
            mma_tf32(d, da + adv, dbl + adv, idesc, 1u);
          }
        }
        mma_commit(&empty[s]);
        if (kt % CH == CH - 1 || kt == nk - 1) mma_commit(&tfull[b]);
      }
    }
  } else {
    // warps 2..5
    const int cw = warp - 2;  // 0..3
    const int lg = warp & 3;  // TMEM lanes 32*lg .. +31 = tile rows
    float acc[BN];
#pragma unroll
    for (int j = 0; j < BN; ++j) acc[j] = 0.f;
    int next = 0;  // next chunk to read out
    bool ok = true;
    // add chunk c's TMEM buffer into acc and release the buffer
    auto drain = [&](int c) -> bool {
      const int b = c & 1;
      if (!mbar_wait(&tfull[b], (uint32_t)((c >> 1) & 1), args.status)) return false;
      tc_fence_after();
#pragma unroll
      for (int cc = 0; cc < BN; cc += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(b * BN + cc), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[cc + j] += v[j];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[b]);
      return true;
    };
    if (SPLIT3) {
      const int t = cw * 32 + lane;
      for (int kt = 0; kt < nk && ok; ++kt) {
        const int s = kt % STAGES, u = kt / STAGES;
        if (!mbar_wait(&full[s], (uint32_t)(u & 1), args.status)) break;
        unsigned char* st = smem + s * STAGE_BYTES;
        float4* a = (float4*)st;
        float4* b = (float4*)(st + A_BYTES);
        float4* alo = (float4*)(st + A_BYTES + B_BYTES);
        float4* blo = (float4*)(st + 2 * A_BYTES + B_BYTES);
        for (int i = t; i < (int)(A_BYTES / 16); i += 128) {
          const float4 x = a[i];
          const float4 h = make_float4(tf32_trunc(x.x), tf32_trunc(x.y), tf32_trunc(x.z), tf32_trunc(x.w));
          a[i] = h;
          alo[i] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        }
        for (int i = t; i < (int)(B_BYTES / 16); i += 128) {
          const float4 x = b[i];
          const float4 h = make_float4(tf32_trunc(x.x), tf32_trunc(x.y), tf32_trunc(x.z), tf32_trunc(x.w));
          b[i] = h;
          blo[i] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[s]);
        // the chunk before the one this slice completes is long done
        if (kt % CH == CH - 1)
          while (next < kt / CH && ok) ok = drain(next++);
      }
    }
    while (next < nch && ok) ok = drain(next++);
    // Epilogue (one row per thread).
    if (ok) {
      const int64_t row = m0 + lg * 32 + lane;
      float* C = args.C + (args.mode == 0 ? (int64_t)blockIdx.z * args.split_stride : 0);
      if (row < args.M) {
#pragma unroll
        for (int j = 0; j < BN; ++j) {
          const int64_t col = n0 + j;
          if (col < args.N) {
            float* p = C + row + col * args.ldc;
            if (args.mode == 0) *p = acc[j];
            else *p -= acc[j];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN))
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Persistent update C (M x N) -= A^T B for a short contraction (K = 128 in the
// outer-block update), operands already split into TF32 high/low arrays by
// the kernels that produce them.  One CTA per SM walks output tiles
// t = blockIdx.x, +gridDim.x, ... (m fastest, so concurrent tiles share the
// B tile in L2).  Warp 0 streams operand slices with TMA; warp 1 issues the
// MMAs into one of two TMEM accumulators (128 columns each); warps 4-11 drain
// the other accumulator meanwhile: each thread owns one row and 64 columns of
// the tile, issues its 64 loads of C at once, subtracts the accumulator and
// stores.  So a tile's epilogue overlaps the next tile's MMAs, and C's load
// latency is paid once per tile, not once per column.
// ---------------------------------------------------------------------------
constexpr int kUpdThreads = 384;
constexpr size_t kUpdCbufBytes = (size_t)256 * 64 * sizeof(float);  // 64 columns per epilogue thread

struct UpdArgs {
  int64_t M, N, K;
  // tile t -> (row tile, column tile) (see update_tile)
  float* C;
  int64_t ldc;
  int64_t mtiles, ntiles;
  int* status;
};

// Output tile t of the persistent update -> its first row m0 and column n0.
// Row tiles are taken in bands of G = gridDim.x: inside a band, tile
// t = band_start + c + i*G goes to row (c + i*G) % R and column
// (c + i*G) / R, R the band's rows.  With full bands every CTA keeps one row
// tile (its slice of V) and walks the columns in step with the others, so
// each V tile is read from DRAM once per band and each W' tile once per
// band, both while they are hot in L2; a row-major walk instead re-reads all
// of V (up to 0.28 GB) for every column tile.
__device__ __forceinline__ void update_tile(int64_t t, int64_t mtiles, int64_t ntiles, int64_t G, int64_t& m0,
                                            int64_t& n0) {
  // 32-bit index arithmetic (the host keeps the tile count below 2^31):
  // 64-bit divisions cost more than the rest of a tile's epilogue
  const uint32_t tt = (uint32_t)t, g = (uint32_t)G, nt = (uint32_t)ntiles, mt = (uint32_t)mtiles;
  const uint32_t band = tt / (g * nt), local = tt - band * g * nt;
  const uint32_t rows = mt - band * g < g ? mt - band * g : g;
  m0 = (int64_t)(band * g + local % rows) * kBM;
  n0 = (int64_t)(local / rows) * kBM;
}

template <bool SPLIT3, int STAGES>
__global__ void __launch_bounds__(kUpdThreads, 1)
    k_tc_update(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, UpdArgs args) {
  constexpr uint32_t TILE = kBM * kBK * 4;  // 16 KB: 128 rows x 32 floats
  constexpr uint32_t STAGE_BYTES = TILE * (SPLIT3 ? 4 : 2);
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = (uint32_t*)(tempty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ntile = args.mtiles * args.ntiles;
  const int nk = (int)((args.K + kBK - 1) / kBK);

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
        update_tile(t, args.mtiles, args.ntiles, gridDim.x, m0l, n0l);
        const int m0 = (int)m0l, n0 = (int)n0l;
        for (int ks = 0; ks < nk; ++ks, ++g) {
          const int s = (int)(g % STAGES);
          const int64_t u = g / STAGES;
          if (u > 0 && !mbar_wait(&empty[s], (uint32_t)((u - 1) & 1), args.status)) { ok = false; break; }
          unsigned char* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          const int x = ks * kBK;
          tma_load_2d(st, &tmAh, x, m0, &full[s]);
          tma_load_2d(st + TILE, &tmBh, x, n0, &full[s]);
          if (SPLIT3) {
            tma_load_2d(st + 2 * TILE, &tmAl, x, m0, &full[s]);
            tma_load_2d(st + 3 * TILE, &tmBl, x, n0, &full[s]);
          }
        }
      }
      if (!ok) {
        // Error exit: let the copies already issued land before the CTA ends.
        for (int64_t q = (g > STAGES ? g - STAGES : 0); q < g; ++q)
          mbar_wait(&full[q % STAGES], (uint32_t)((q / STAGES) & 1), args.status, false);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kBM >> 3) << 17) |
                             ((uint32_t)(kBM >> 4) << 24);
      int64_t g = 0;
      int it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntile && ok; t += gridDim.x, ++it) {
        const int acc = it & 1, ua = it >> 1;
        if (ua > 0 && !mbar_wait(&tempty[acc], (uint32_t)((ua - 1) & 1), args.status)) { ok = false; break; }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * kBM);
        for (int ks = 0; ks < nk; ++ks, ++g) {
          const int s = (int)(g % STAGES);
          const int64_t u = g / STAGES;
          if (!mbar_wait(&full[s], (uint32_t)(u & 1), args.status)) { ok = false; break; }
          tc_fence_after();
          unsigned char* st = smem + s * STAGE_BYTES;
          const uint64_t dah = sdesc_sw128(st), dbh = sdesc_sw128(st + TILE);
#pragma unroll
          for (int kk = 0; kk < kBK / 8; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 2);
            mma_tf32(d, dah + adv, dbh + adv, idesc, (ks > 0 || kk > 0) ? 1u : 0u);
            if (SPLIT3) {
              const uint64_t dal = sdesc_sw128(st + 2 * TILE), dbl = sdesc_sw128(st + 3 * TILE);
              mma_tf32(d, dal + adv, dbh + adv, idesc, 1u);
              mma_tf32(d, dah + adv, dbl + adv, idesc, 1u);
            }
          }
          mma_commit(&empty[s]);
        }
        mma_commit(&tfull[acc]);
      }
    }
  } else if (warp >= 4) {
    const int lg = warp & 3, half = (warp - 4) >> 2;
    // this thread's slice of the next tile's C (row, 64 columns) is copied
    // into its own part of cbuf (element j at j * 256 + et) while the current
    // tile waits for its accumulator and is stored
    const int et = threadIdx.x - 128;
    float* cbuf = (float*)(smem + STAGES * STAGE_BYTES + 256);
    const int64_t ldc = args.ldc;
    auto prefetch = [&](int64_t t) {
      int64_t m0, n0;
      update_tile(t, args.mtiles, args.ntiles, gridDim.x, m0, n0);
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
      update_tile(t, args.mtiles, args.ntiles, gridDim.x, m0, n0);
      const int64_t row = m0 + lg * 32 + lane;
      const int64_t c0 = n0 + half * 64;
      const bool rok = row < args.M;
      float c[64];
      cp_async_wait_all();
#pragma unroll
      for (int j = 0; j < 64; ++j) c[j] = cbuf[j * 256 + et];
      if (t + gridDim.x < ntile) prefetch(t + gridDim.x);
      if (!mbar_wait(&tfull[acc], (uint32_t)(ua & 1), args.status)) {
        cp_async_wait_all();
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(acc * kBM + half * 64 + q * 16), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) c[q * 16 + i] -= v[i];
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
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

// 2-D FP32 tensor: d0 contiguous elements per column, d1 columns, column
// stride ld elements; boxes of box0 x box1 with 128-byte swizzle.
bool make_map(CUtensorMap* m, const float* base, uint64_t d0, uint64_t d1, uint64_t ld, uint32_t box0,
              uint32_t box1) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {d0, d1};
  cuuint64_t strides[1] = {ld * 4};
  cuuint32_t box[2] = {box0, box1};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int STAGES, bool SPLIT3>
ct_status launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& a, int splits, cudaStream_t s) {
  constexpr size_t STAGE_BYTES = (size_t)(kBM + BN) * kBK * 4 * (SPLIT3 ? 2 : 1);
  const size_t smem = STAGES * STAGE_BYTES + 1024 + 256;
  static bool attr_done = false;
  if (!attr_done) {
    CT_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm_tn<BN, STAGES, SPLIT3>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_done = true;
  }
  const dim3 grid((unsigned)((a.M + kBM - 1) / kBM), (unsigned)((a.N + BN - 1) / BN), (unsigned)splits);
  k_tc_gemm_tn<BN, STAGES, SPLIT3><<<grid, kThreads, smem, s>>>(ma, mb, a);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

template <bool SPLIT3, int STAGES>
ct_status launch_upd(const CUtensorMap* maps, const UpdArgs& a, int sms, cudaStream_t s) {
  constexpr size_t STAGE_BYTES = (size_t)kBM * kBK * 4 * (SPLIT3 ? 4 : 2);
  // operand stages, alignment slack, barriers, and the epilogue's C buffer
  const size_t smem = STAGES * STAGE_BYTES + 1024 + 256 + kUpdCbufBytes;
  static bool attr_done = false;
  if (!attr_done) {
    CT_CUDA_TRY(cudaFuncSetAttribute(k_tc_update<SPLIT3, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    attr_done = true;
  }
  const int64_t tiles = a.mtiles * a.ntiles;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
  k_tc_update<SPLIT3, STAGES><<<grid, kUpdThreads, smem, s>>>(maps[0], maps[1], maps[2], maps[3], a);
  CT_LAUNCH_CHECK();
  return CT_OK;
}

}  // namespace

// C (M x N) -= A^T B with pre-split operands (Ah/Al: K x M, Bh/Bl: K x N,
// column-major FP32, lda/ldb multiples of 4); Al/Bl ignored unless split3.
ct_status tc_update_presplit(const float* Ah, const float* Al, int64_t lda, const float* Bh, const float* Bl,
                             int64_t ldb, int64_t M, int64_t N, int64_t K, float* C, int64_t ldc, bool split3,
                             int sms, int* status, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return CT_OK;
  if (!Ah || !Bh || !C || (split3 && (!Al || !Bl)) || lda < K || ldb < K || ldc < M) return CT_ERR_INVALID;
  if (((uintptr_t)Ah & 15) || ((uintptr_t)Bh & 15) || (split3 && (((uintptr_t)Al & 15) || ((uintptr_t)Bl & 15))) ||
      (lda & 3) || (ldb & 3))
    return CT_ERR_INVALID;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return CT_ERR_INVALID;
  CUtensorMap maps[4];
  if (!make_map(&maps[0], Ah, (uint64_t)K, (uint64_t)M, (uint64_t)lda, kBK, kBM)) return CT_ERR_CUDA;
  if (!make_map(&maps[2], Bh, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, kBK, kBM)) return CT_ERR_CUDA;
  if (split3) {
    if (!make_map(&maps[1], Al, (uint64_t)K, (uint64_t)M, (uint64_t)lda, kBK, kBM)) return CT_ERR_CUDA;
    if (!make_map(&maps[3], Bl, (uint64_t)K, (uint64_t)N, (uint64_t)ldb, kBK, kBM)) return CT_ERR_CUDA;
  } else {
    maps[1] = maps[0];
    maps[3] = maps[2];
  }
  UpdArgs a;
  a.M = M;
  a.N = N;
  a.K = K;
  a.C = C;
  a.ldc = ldc;
  a.mtiles = (M + kBM - 1) / kBM;
  a.ntiles = (N + kBM - 1) / kBM;
  if (a.mtiles * a.ntiles + sms > INT32_MAX) return CT_ERR_INVALID;  // 32-bit tile indices
  a.status = status;
  LaunchScope ls(K_TC_UPDATE, s, 2.0 * M * N * K, 4.0 * ((double)K * (M + N) * (split3 ? 2 : 1) + 2.0 * M * N));
  if (split3) return launch_upd<true, 2>(maps, a, sms, s);
  return launch_upd<false, 4>(maps, a, sms, s);
}

// C (M x N) = / -= A^T B on the tensor cores; see the file comment.
ct_status tc_gemm_tn(const float* A, int64_t lda, const float* B, int64_t ldb, int64_t M, int64_t N,
                     int64_t K, float* C, int64_t ldc, int64_t split_stride, int mode, int splits,
                     bool split3, int* status, cudaStream_t s) {
  if (M <= 0 || N <= 0) return CT_OK;
  if (!A || !B || !C || K < 0 || lda < K || ldb < K || ldc < M) return CT_ERR_INVALID;
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || (lda & 3) || (ldb & 3)) return CT_ERR_INVALID;
  if (M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return CT_ERR_INVALID;
  if (splits < 1) splits = 1;
  int64_t chunk = (K + splits - 1) / splits;
  chunk = (chunk + kBK - 1) / kBK * kBK;
  if (chunk < kBK) chunk = kBK;
  splits = (int)((K + chunk - 1) / chunk);
  if (splits < 1) splits = 1;
  if (mode == 0 && splits > 1 && split_stride < ldc * N) return CT_ERR_INVALID;
  if (mode != 0 && splits > 1) return CT_ERR_INVALID;  // in-place subtraction must not be split
  CUtensorMap ma, mb;
  const uint64_t kd = K > 0 ? (uint64_t)K : 1;
  constexpr int BN = 128;
  if (!make_map(&ma, A, kd, (uint64_t)M, (uint64_t)lda, kBK, kBM)) return CT_ERR_CUDA;
  if (!make_map(&mb, B, kd, (uint64_t)N, (uint64_t)ldb, kBK, BN)) return CT_ERR_CUDA;
  TcArgs a;
  a.M = M;
  a.N = N;
  a.K = K;
  a.k_chunk = chunk;
  a.ch = kAccChunkSlices;
  a.C = C;
  a.ldc = ldc;
  a.split_stride = split_stride;
  a.mode = mode;
  a.status = status;
  LaunchScope ls(K_TC_GEMM, s, 2.0 * M * N * K,
                 4.0 * ((double)K * (M + N) + (mode == 0 ? 1.0 : 2.0) * M * N));
  if (split3) return launch_tc<BN, 3, true>(ma, mb, a, splits, s);
  return launch_tc<BN, 6, false>(ma, mb, a, splits, s);
}

}  // namespace ctqr
