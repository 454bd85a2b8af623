// The surrogate's large GEMMs on the 5th-generation tensor cores (sm_103a):
// C[m, n] = sum_k A[m][k] B[n][k] (+ bias[n], GELU on the bfloat16 copy),
// bfloat16 operands, FP32 accumulation, for M up to millions of rows (16 per
// env, or 96 for the edge MLP), N <= 128 and K <= 128 a multiple of 8: the
// shapes of the network's layers and of their input gradients.
//
//   operands  cp.async.bulk.tensor (TMA) 2D tiles into shared memory with the
//             128-byte swizzle, K-major: a 128-row tile of A per stage (two
//             stages), the whole of B once per CTA; K past the tensor's end
//             and rows past M are filled with zeros by the copy engine
//   MMA       tcgen05.mma kind::f16 (M = 128, N = N rounded up to 16, K = 16
//             per instruction; K = 8 reads zeros in 8..15), issued by one
//             thread, accumulating in TMEM:
//             two 128-column accumulators, so the MMAs of tile i + 1 run
//             while the twelve warps read tile i back
//   epilogue  tcgen05.ld (32 lanes x 32 bits: thread t of warp w owns TMEM
//             lane 32 (w % 4) + t, i.e. one output row, and every third
//             16-column chunk from chunk w / 4 on: three warps per lane
//             quarter), bias, GELU (the same values as the warp-mma
//             path's); FP32 and bfloat16 outputs staged per warp in shared
//             memory (32 rows x 32 bytes) and written by TMA tensor stores
//   waits     every mbarrier wait is bounded (about a second); a CTA whose
//             wait runs out sets VMAS_DEVERR_TIMEOUT in the error word, waits
//             (bounded) for its copies in flight, frees its TMEM and returns
//
// Persistent: a grid of at most two CTAs per SM (the shared-memory request is
// padded so that no third fits, which keeps the two 256-column TMEM
// allocations of an SM within its 512 columns) walks the 128-row tiles.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "mbar.cuh"
#include "surrogate.cuh"
#include "vmas.h"

namespace vmas {
namespace sur {

constexpr int kTcM = 128;                // rows per tile (the MMA's M)
constexpr int kTcAtom = kTcM * 128;      // bytes of a 64-wide K slice of a tile
constexpr int kTcCols = 256;             // TMEM columns per CTA (two accumulators)
constexpr int kTcMinSmem = 80 * 1024;    // at most two CTAs per SM
constexpr int kTcWaitTries = 1 << 20;    // polls of at most ~1 us each
constexpr int kTcThreads = 384;          // 12 warps: three per TMEM lane quarter in the epilogue

struct TcGemmArgs {
  int M, N, K;         // N <= 128, K <= 128, K % 8 == 0
  int n_pad;           // N rounded up to 16: the MMA's N and B's box height
  int katoms;          // ceil(K / 64): 64-element K slices per tile
  const float *bias;   // [N] or null
  int act;             // 1: GELU on the bfloat16 output
  float *out_f32;      // [M][ldc_f] or null
  int ldc_f;
  bf16 *out_bf;        // [M][ldc_b] or null
  int ldc_b;
  int *err;            // device error word
  int vec_f, vec_b;    // 16-byte stores allowed (aligned bases, ldc_f % 4, ldc_b % 8)
  int tma_st;          // outputs written by TMA stores (tensor maps tmC, tmCb valid)
  // test hook: extra transaction bytes every A-tile barrier waits for, which
  // no copy delivers, so that its bounded wait runs out (0 in normal use)
  uint32_t extra_tx;
};

// Output staging for TMA stores: per warp, 32 rows x 32 bytes (a 16-column
// bfloat16 chunk, or half of a 16-column FP32 chunk), 128-byte aligned after
// the barriers.
constexpr int kTcStage = 32 * 32;
__host__ __device__ inline int tc_stage_offset(int katoms, int n_pad) {
  return (2 * katoms * kTcAtom + katoms * n_pad * 128 + 64 + 127) & ~127;
}
__host__ __device__ inline int tc_smem_bytes(int katoms, int n_pad) {
  const int b = 1024 + tc_stage_offset(katoms, n_pad) + (kTcThreads / 32) * kTcStage;
  return b < kTcMinSmem ? kTcMinSmem : b;
}

// TMA tensor store of a 2D box from shared memory (bulk group of the
// issuing thread), the group's commit, and the waits for its shared-memory
// reads and for its completion.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(src), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout: 8-row groups 1024 bytes apart (stride byte offset), the
// leading byte offset unused for this layout (1), descriptor version 1,
// swizzle mode 2 (128 B).  `addr` is the shared-memory byte address of the
// K slice's first element; the slice's 1024-byte atom must be aligned.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                   // leading byte offset (16 B, unused)
  d |= (uint64_t)(1024u >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1u << 46;                   // version
  d |= (uint64_t)2u << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, bfloat16 A and B,
// both K-major, N >> 3 and M >> 4.
__host__ __device__ inline uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__global__ void __launch_bounds__(kTcThreads, 2)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmCb,
                   const TcGemmArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int KA = g.katoms;
  unsigned char *sA = base;                        // [2 stages][KA atoms][128 rows][128 B]
  unsigned char *sB = base + 2 * KA * kTcAtom;     // [KA atoms][n_pad rows][128 B]
  unsigned long long *bar =
      reinterpret_cast<unsigned long long *>(sB + KA * g.n_pad * 128);  // full[2], done[2], bfull
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 5);
  unsigned char *stg = base + tc_stage_offset(KA, g.n_pad) + warp * kTcStage;  // this warp's
  const uint32_t full0 = smem_u32(&bar[0]), done0 = smem_u32(&bar[2]), bfull = smem_u32(&bar[4]);
  const int tiles = (g.M + kTcM - 1) / kTcM;
  const int mine = tiles > (int)blockIdx.x ? (tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const uint32_t a_bytes = (uint32_t)(KA * kTcAtom), b_bytes = (uint32_t)(KA * g.n_pad * 128);
  const int ksteps = (g.K + 15) / 16;  // K = 8: the copy engine zero-fills 8..15
  const uint32_t idesc = tc_idesc(kTcM, g.n_pad);

  // the bias, zero past N, for the TMA-store epilogue's 16-byte reads
  __shared__ __align__(16) float s_bias[128];
  for (int q = tid; q < 128; q += blockDim.x) s_bias[q] = g.bias && q < g.N ? g.bias[q] : 0.f;
  if (tid == 0) {
    for (int q = 0; q < 5; ++q) mbar_init(smem_u32(&bar[q]), 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // loads and MMA commits issued per stage (thread 0's counts)
  int issued[2] = {0, 0}, committed[2] = {0, 0};
  auto load_a = [&](int i) {  // thread 0: tile of local index i into stage i & 1
    const int s = i & 1, row = ((int)blockIdx.x + i * (int)gridDim.x) * kTcM;
    mbar_expect_tx(full0 + 8 * s, a_bytes + g.extra_tx);
    for (int a = 0; a < KA; ++a)
      tma_load_2d(smem_u32(sA + (s * KA + a) * kTcAtom), &tmA, 64 * a, row, full0 + 8 * s);
    ++issued[s];
  };
  if (tid == 0 && mine > 0) {
    mbar_expect_tx(bfull, b_bytes);
    for (int a = 0; a < KA; ++a)
      tma_load_2d(smem_u32(sB + a * g.n_pad * 128), &tmB, 64 * a, 0, bfull);
    load_a(0);
    if (mine > 1) load_a(1);
  }
  bool failed = false;  // thread 0: a wait of its own ran out
  auto issue = [&](int i) {  // thread 0: the MMAs of local tile i, committed to done[i & 1]
    const int s = i & 1;
    if (i == 0 && !mbar_wait(bfull, 0, kTcWaitTries)) { failed = true; return; }
    if (!mbar_wait(full0 + 8 * s, (uint32_t)((i >> 1) & 1), kTcWaitTries)) { failed = true; return; }
    tc_fence_after();
    const uint32_t a0 = smem_u32(sA + s * KA * kTcAtom), b0 = smem_u32(sB);
    for (int j = 0; j < ksteps; ++j) {
      const uint32_t off_a = (uint32_t)((j >> 2) * kTcAtom + (j & 3) * 32);
      const uint32_t off_b = (uint32_t)((j >> 2) * g.n_pad * 128 + (j & 3) * 32);
      tc_mma(tmem + (uint32_t)(s * 128), tc_desc(a0 + off_a), tc_desc(b0 + off_b), idesc,
             j > 0 ? 1u : 0u);
    }
    tc_commit(done0 + 8 * s);
    ++committed[s];
  };
  if (tid == 0 && mine > 0) issue(0);

  for (int i = 0; i < mine; ++i) {
    const int s = i & 1;
    if (tid == 0 && i + 1 < mine && !failed) issue(i + 1);
    const bool late = !mbar_wait(done0 + 8 * s, (uint32_t)((i >> 1) & 1), kTcWaitTries);
    if (__syncthreads_or(late || failed)) {
      failed = true;
      break;
    }
    tc_fence_after();
    // stage s is free once its MMAs have completed: prefetch tile i + 2
    if (tid == 0 && i + 2 < mine) load_a(i + 2);
    // warp w reads TMEM lane quarter w % 4 (its rows) and every third
    // 16-column chunk, starting at chunk w / 4
    const int quarter = warp & 3;
    const int row = ((int)blockIdx.x + i * (int)gridDim.x) * kTcM + quarter * 32 + lane;
    const uint32_t tbase = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(s * 128);
    for (int c0 = 16 * (warp >> 2); c0 < g.n_pad; c0 += 16 * (kTcThreads / 128)) {
      float v[16];
      tc_ld16(tbase + (uint32_t)c0, v);
      if (g.tma_st) {
        // the whole warp: bias, then each output through the warp's staging
        // rows (lane l: row l, 32 bytes) and one TMA store of 32 rows x 32
        // bytes, which the copy engine clips at M and N
        if (g.bias) {  // (no bias: nothing added, so -0 stays -0)
          const float4 *b4 = reinterpret_cast<const float4 *>(s_bias + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 b = b4[q];
            v[4 * q] += b.x;
            v[4 * q + 1] += b.y;
            v[4 * q + 2] += b.z;
            v[4 * q + 3] += b.w;
          }
        }
        const int y0 = row - lane;
        const bool any = y0 < g.M;  // the warp's rows are not all past M
        uint4 *srow = reinterpret_cast<uint4 *>(stg + lane * 32);
        if (g.out_f32 && any) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            if (c0 + 8 * h < g.N) {  // the same for the whole warp
              if (lane == 0) bulk_wait_read();  // the buffer's previous store has read it
              __syncwarp();
              srow[0] = make_uint4(__float_as_uint(v[8 * h]), __float_as_uint(v[8 * h + 1]),
                                   __float_as_uint(v[8 * h + 2]), __float_as_uint(v[8 * h + 3]));
              srow[1] = make_uint4(__float_as_uint(v[8 * h + 4]), __float_as_uint(v[8 * h + 5]),
                                   __float_as_uint(v[8 * h + 6]), __float_as_uint(v[8 * h + 7]));
              fence_proxy_async_smem();
              __syncwarp();
              if (lane == 0) {
                tma_store_2d(&tmC, smem_u32(stg), c0 + 8 * h, y0);
                bulk_commit();
              }
            }
          }
        }
        if (g.out_bf && any) {
          uint32_t w[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float2 x = make_float2(v[2 * q], v[2 * q + 1]);
            if (g.act) x = gelu2(x);
            const __nv_bfloat162 hh = __floats2bfloat162_rn(x.x, x.y);
            w[q] = *reinterpret_cast<const uint32_t *>(&hh);
          }
          if (lane == 0) bulk_wait_read();
          __syncwarp();
          srow[0] = make_uint4(w[0], w[1], w[2], w[3]);
          srow[1] = make_uint4(w[4], w[5], w[6], w[7]);
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_2d(&tmCb, smem_u32(stg), c0, y0);
            bulk_commit();
          }
        }
      } else if (row < g.M && c0 + 16 <= g.N) {
        // a full 16-column block of this row
#pragma unroll
        for (int q = 0; q < 16; ++q)
          if (g.bias) v[q] += g.bias[c0 + q];
        if (g.out_f32) {
          float *o = g.out_f32 + (size_t)row * g.ldc_f + c0;
          if (g.vec_f) {
#pragma unroll
            for (int q = 0; q < 16; q += 4)
              *reinterpret_cast<float4 *>(o + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) o[q] = v[q];
          }
        }
        if (g.out_bf) {
          bf16 *o = g.out_bf + (size_t)row * g.ldc_b + c0;
          uint32_t w[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float2 x = make_float2(v[2 * q], v[2 * q + 1]);
            if (g.act) x = gelu2(x);
            const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
            w[q] = *reinterpret_cast<const uint32_t *>(&h);
          }
          if (g.vec_b) {
            reinterpret_cast<uint4 *>(o)[0] = make_uint4(w[0], w[1], w[2], w[3]);
            reinterpret_cast<uint4 *>(o)[1] = make_uint4(w[4], w[5], w[6], w[7]);
          } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              o[2 * q] = __ushort_as_bfloat16((unsigned short)(w[q] & 0xffffu));
              o[2 * q + 1] = __ushort_as_bfloat16((unsigned short)(w[q] >> 16));
            }
          }
        }
      } else if (row < g.M) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int n = c0 + q;
          if (n < g.N) {
            float x = v[q];
            if (g.bias) x += g.bias[n];
            if (g.out_f32) g.out_f32[(size_t)row * g.ldc_f + n] = x;
            if (g.out_bf) g.out_bf[(size_t)row * g.ldc_b + n] = __float2bfloat16_rn(g.act ? gelu(x) : x);
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // both TMEM accumulators' readers are done before the next MMAs
  }
  if (g.tma_st && lane == 0) bulk_wait_all();  // this warp's stores are done with its buffer
  if (failed) {
    if (tid == 0) {
      atomicOr(g.err, VMAS_DEVERR_TIMEOUT);
      // wait (bounded) for the copies still in flight into this CTA's memory
      // and for the MMAs still reading it and writing TMEM
      for (int s = 0; s < 2; ++s) {
        if (issued[s] > 0) mbar_wait(full0 + 8 * s, (uint32_t)((issued[s] - 1) & 1), kTcWaitTries);
        if (committed[s] > 0)
          mbar_wait(done0 + 8 * s, (uint32_t)((committed[s] - 1) & 1), kTcWaitTries);
      }
      if (mine > 0) mbar_wait(bfull, 0, kTcWaitTries);
    }
    __syncthreads();
  }
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols)
                 : "memory");
  }
}

// ---------------------------------------------------------- weight gradients
// C[m][n] = sum_k A[k][m] B[k][n] for the weight gradients of the network's
// layers: M, N <= 128 (a layer's output and input widths), K = the rows of a
// batch (millions).  Both operands are read as they lie in memory, rows of
// the batch outermost: the MN-major operand layout of tcgen05.mma (both
// transpose bits of the instruction descriptor set).
//
//   split K    CTA z sums the 64-row blocks [z kb, (z + 1) kb) of K (rows
//              past K read as zeros) into a TMEM accumulator and writes its
//              partial [M][N] to part + z M N; sum_partials_kernel adds them
//   operands   per 64-row block, TMA tiles of 64 rows x 64 columns with the
//              128-byte swizzle: two for A (columns 0-63, 64-127), one or two
//              for B; the MN-major layout is then: a row of 64 elements per
//              128 bytes, 8-row groups 1024 bytes apart (stride byte offset),
//              the second 64 columns one tile (8 KB) further (leading byte
//              offset); three stages in a ring, each freed by the commit of
//              the MMAs that read it
//   MMA        M = 128 (A's columns; when M <= 64 the upper half of A stays
//              zero), N = 64 or 128, K = 16 per instruction: 4 per block,
//              each 16 rows (2 KB) further into the tiles
//   waits      bounded as in gemm_tc_kernel (error word, drain, TMEM freed)
constexpr int kWgStages = 3;
constexpr int kWgTile = 64 * 128;                 // bytes of a 64 x 64 bfloat16 tile
constexpr int kWgStage = 4 * kWgTile;             // A (2 tiles) + B (2 tiles)
constexpr int kWgCols = 128;                      // TMEM columns (one accumulator)

struct WgradArgs {
  int M, N;        // M, N <= 128
  int n_mma;       // 64 or 128
  int kb;          // 64-row blocks per CTA
  int nblocks;     // 64-row blocks of K
  float *part;     // [gridDim.x][M][N]
  int *err;
  int vec;         // N % 4 == 0: 16-byte partial stores
  uint32_t extra_tx;  // test hook, as in TcGemmArgs (0 in normal use)
};

__host__ __device__ inline int wgrad_smem_bytes() {
  // 1 KB alignment, the stages, 8 KB of slack past the last tile, barriers
  return 1024 + kWgStages * kWgStage + 8 * 1024 + 128;
}

// Shared-memory descriptor of an MN-major operand in the 128-byte swizzled
// layout: 64-element rows 128 B apart, 8-row groups 1024 B apart (stride
// byte offset), the next 64 columns `lbo` bytes on (leading byte offset).
__device__ __forceinline__ uint64_t tc_desc_mn(uint32_t addr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

__global__ void __launch_bounds__(128, 2)
    wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const WgradArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned long long *bar = reinterpret_cast<unsigned long long *>(
      base + kWgStages * kWgStage + 8 * 1024);  // full[S], empty[S]
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2 * kWgStages);
  const uint32_t full0 = smem_u32(&bar[0]), empty0 = smem_u32(&bar[kWgStages]);
  const int b0 = (int)blockIdx.x * g.kb;
  const int nb = max(0, min(g.kb, g.nblocks - b0));  // this CTA's blocks
  const bool two_a = g.M > 64, two_b = g.n_mma > 64;
  const uint32_t bytes = (uint32_t)((two_a ? 2 : 1) + (two_b ? 2 : 1)) * kWgTile;
  const uint32_t idesc = tc_idesc(kTcM, g.n_mma) | (1u << 15) | (1u << 16);

  if (!two_a) {  // the upper 64 columns of A are zero in every stage
    for (int s = 0; s < kWgStages; ++s)
      for (int q = tid; q < kWgTile / 16; q += blockDim.x)
        reinterpret_cast<uint4 *>(base + s * kWgStage + kWgTile)[q] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < 2 * kWgStages; ++q) mbar_init(smem_u32(&bar[q]), 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kWgCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  bool failed = false;
  int loaded[kWgStages] = {}, committed[kWgStages] = {};
  if (tid == 0) {
    auto load = [&](int b) {  // block b of this CTA into stage b % S
      const int s = b % kWgStages, row = 64 * (b0 + b);
      unsigned char *st = base + s * kWgStage;
      mbar_expect_tx(full0 + 8 * s, bytes + g.extra_tx);
      tma_load_2d(smem_u32(st), &tmA, 0, row, full0 + 8 * s);
      if (two_a) tma_load_2d(smem_u32(st + kWgTile), &tmA, 64, row, full0 + 8 * s);
      tma_load_2d(smem_u32(st + 2 * kWgTile), &tmB, 0, row, full0 + 8 * s);
      if (two_b) tma_load_2d(smem_u32(st + 3 * kWgTile), &tmB, 64, row, full0 + 8 * s);
      ++loaded[s];
    };
    for (int b = 0; b < nb && b < kWgStages; ++b) load(b);
    for (int b = 0; b < nb; ++b) {
      const int s = b % kWgStages;
      const uint32_t par = (uint32_t)((b / kWgStages) & 1);
      if (!mbar_wait(full0 + 8 * s, par, kTcWaitTries)) { failed = true; break; }
      tc_fence_after();
      const uint32_t a0 = smem_u32(base + s * kWgStage), bb0 = a0 + 2 * kWgTile;
      for (int j = 0; j < 4; ++j)
        tc_mma(tmem, tc_desc_mn(a0 + 2048u * j, kWgTile), tc_desc_mn(bb0 + 2048u * j, kWgTile),
               idesc, (b > 0 || j > 0) ? 1u : 0u);
      tc_commit(empty0 + 8 * s);
      ++committed[s];
      if (b + kWgStages < nb) {
        if (!mbar_wait(empty0 + 8 * s, par, kTcWaitTries)) { failed = true; break; }
        load(b + kWgStages);
      }
    }
    // the last block's MMAs complete before the accumulator is read
    if (!failed && nb > 0) {
      const int s = (nb - 1) % kWgStages;
      if (!mbar_wait(empty0 + 8 * s, (uint32_t)(((nb - 1) / kWgStages) & 1), kTcWaitTries))
        failed = true;
    }
    if (failed) {
      atomicOr(g.err, VMAS_DEVERR_TIMEOUT);
      for (int s = 0; s < kWgStages; ++s) {
        if (loaded[s] > 0) mbar_wait(full0 + 8 * s, (uint32_t)((loaded[s] - 1) & 1), kTcWaitTries);
        if (committed[s] > 0)
          mbar_wait(empty0 + 8 * s, (uint32_t)((committed[s] - 1) & 1), kTcWaitTries);
      }
    }
  }
  tc_fence_before();
  failed = __syncthreads_or(failed);
  tc_fence_after();
  if (!failed) {
    // thread t of warp w: accumulator row m = 32 w + t, 16 columns at a time
    const int m = warp * 32 + lane;
    float *o = g.part + ((size_t)blockIdx.x * g.M + m) * g.N;
    for (int c0 = 0; c0 < g.n_mma; c0 += 16) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (nb == 0) {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = 0.f;
      }
      if (m < g.M) {
        if (g.vec && c0 + 16 <= g.N) {
#pragma unroll
          for (int q = 0; q < 16; q += 4)
            *reinterpret_cast<float4 *>(o + c0 + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (c0 + q < g.N) o[c0 + q] = v[q];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWgCols)
                 : "memory");
  }
}

}  // namespace sur
}  // namespace vmas
