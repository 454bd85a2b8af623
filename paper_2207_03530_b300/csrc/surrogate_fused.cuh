// Fused inference of the learned surrogate (sm_103a): one warp per env, the
// 16 agents of an env being the 16 rows of every warp-level bfloat16 mma
// (m16n8k16, FP32 accumulation).  Features, the edge MLP for each neighbour
// slot, the masked sum, the node MLP, the prediction and the overlap check
// run without leaving the SM; the weights (bfloat16, rows padded by 8
// elements so that ldmatrix phases hit distinct banks) are staged into
// shared memory once per persistent CTA.
//
// Code size matters here: a fully unrolled kernel (every slot, every GELU
// inlined) overflows the instruction cache and stalls on instruction fetch
// most of the time, so the slot loop stays rolled (features of all slots are
// staged in shared memory first) and GELU is one out-of-line routine taking
// two packed pairs.
//
// Arithmetic is that of the layered path (surrogate.cuh): the same rounding
// points, the same k order inside every dot product (k-tiles ascending), the
// same order of the masked sum over slots.
#pragma once

#include "surrogate.cuh"

namespace vmas {
namespace sur {

constexpr int kFusedWarpsPerCta = 16;
// padded row lengths (bfloat16 elements) of the staged weights and of the
// per-warp feature rows
constexpr int kLdE1 = 16 + 8, kLdE2 = 64 + 8, kLdN1 = 80 + 8, kLdN2 = 128 + 8, kLdN3 = 128 + 8;
constexpr int kLdX = 16 + 8;
constexpr int kSmE1 = 0;
constexpr int kSmE2 = kSmE1 + 64 * kLdE1;
constexpr int kSmN1 = kSmE2 + 64 * kLdE2;
constexpr int kSmN2 = kSmN1 + 128 * kLdN1;
constexpr int kSmN3 = kSmN2 + 128 * kLdN2;
constexpr int kSmWeights = kSmN3 + 8 * kLdN3;         // bfloat16 elements
constexpr int kSmBias = 64 + 64 + 128 + 128 + 8;      // floats: be1 be2 b1 b2 b3
// bfloat16 elements per warp: node rows, edge rows per slot, then 16 bytes
// holding the agent of each row
constexpr int kSmWarp = (1 + kK) * 16 * kLdX + 8;
constexpr size_t fused_smem_bytes() {
  return (size_t)kSmWeights * 2 + (size_t)kSmBias * 4 + (size_t)kFusedWarpsPerCta * kSmWarp * 2;
}

struct FusedArgs {
  int E, N, A;
  float *px, *py, *vx, *vy;  // the world's state planes
  const float4 *param;       // {1/m, 1/I, radius, -}
  const float *actions;      // [E][A][3]
  const bf16 *w;             // flat parameters, bfloat16
  const float *p;            // flat parameters, FP32 (biases)
  float *out;                // optional network output [E * 16][8]
  int apply;                 // 1: apply the prediction / list fallback envs
  float limit;
  int *list, *list_len;
};

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// Four 8x8 bfloat16 matrices from shared memory; lane l gives the address
// of row l % 8 of matrix l / 8 and receives (row l / 4, cols 2 (l % 4), +1)
// of each.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16 *p) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

// A fragment (k-tile kk) of 16 rows X with row length ld.
__device__ __forceinline__ void load_a(uint32_t (&a)[4], const bf16 *X, int ld, int kk, int lane) {
  const int m = lane >> 3;
  ldsm_x4(a, X + ((m & 1) * 8 + (lane & 7)) * ld + 16 * kk + (m >> 1) * 8);
}

// B fragments of n-tiles j, j + 1 (k-tile kk) of a weight W [n][k] with row
// length ld: {b0, b1} of tile j, then of tile j + 1.
__device__ __forceinline__ void load_b2(uint32_t (&b)[4], const bf16 *W, int ld, int j, int kk,
                                        int lane) {
  const int m = lane >> 3;
  ldsm_x4(b, W + (8 * (j + (m >> 1)) + (lane & 7)) * ld + 16 * kk + (m & 1) * 8);
}

// B fragments of n-tile 0 for k-tiles kk, kk + 1.
__device__ __forceinline__ void load_b1k2(uint32_t (&b)[4], const bf16 *W, int ld, int kk,
                                          int lane) {
  const int m = lane >> 3;
  ldsm_x4(b, W + (lane & 7) * ld + 16 * (kk + (m >> 1)) + (m & 1) * 8);
}

// bias + GELU on packed pairs, out of line (one copy of the GELU code in the
// kernel); the pairs' dependency chains interleave inside the routine.
// Eight pairs: both pairs of c_i (the two rows of an n-tile fragment) with
// bias b_i.
struct Gelu16 {
  float4 v[4];
};
__device__ __noinline__ Gelu16 gelu_bias16(float4 c0, float4 c1, float4 c2, float4 c3, float2 b0,
                                           float2 b1, float2 b2, float2 b3) {
  const float2 p0 = gelu2(f2_add(make_float2(c0.x, c0.y), b0));
  const float2 p1 = gelu2(f2_add(make_float2(c0.z, c0.w), b0));
  const float2 p2 = gelu2(f2_add(make_float2(c1.x, c1.y), b1));
  const float2 p3 = gelu2(f2_add(make_float2(c1.z, c1.w), b1));
  const float2 p4 = gelu2(f2_add(make_float2(c2.x, c2.y), b2));
  const float2 p5 = gelu2(f2_add(make_float2(c2.z, c2.w), b2));
  const float2 p6 = gelu2(f2_add(make_float2(c3.x, c3.y), b3));
  const float2 p7 = gelu2(f2_add(make_float2(c3.z, c3.w), b3));
  return {{make_float4(p0.x, p0.y, p1.x, p1.y), make_float4(p2.x, p2.y, p3.x, p3.y),
           make_float4(p4.x, p4.y, p5.x, p5.y), make_float4(p6.x, p6.y, p7.x, p7.y)}};
}
// Four pairs: (c0.x, c0.y) with bias b0, (c0.z, c0.w) with b1, (c1.x, c1.y)
// with b2, (c1.z, c1.w) with b3.
struct Gelu8 {
  float4 lo, hi;
};
__device__ __noinline__ Gelu8 gelu_bias8(float4 c0, float4 c1, float2 b0, float2 b1, float2 b2,
                                         float2 b3) {
  const float2 p0 = gelu2(f2_add(make_float2(c0.x, c0.y), b0));
  const float2 p1 = gelu2(f2_add(make_float2(c0.z, c0.w), b1));
  const float2 p2 = gelu2(f2_add(make_float2(c1.x, c1.y), b2));
  const float2 p3 = gelu2(f2_add(make_float2(c1.z, c1.w), b3));
  return {make_float4(p0.x, p0.y, p1.x, p1.y), make_float4(p2.x, p2.y, p3.x, p3.y)};
}

__device__ __forceinline__ float4 f4(const float (&c)[4]) {
  return make_float4(c[0], c[1], c[2], c[3]);
}
__device__ __forceinline__ float2 bias_pair(const float *bias, int n) {
  return *reinterpret_cast<const float2 *>(bias + n);
}

// bias + GELU of the n-tiles 2 kk .. 2 kk + 3 (accumulators c[0..3]),
// rounded into the A fragments of k-tiles kk and kk + 1 of the next layer.
__device__ __forceinline__ void gelu_pack2(uint32_t (&a0)[4], uint32_t (&a1)[4],
                                           const float (&c)[4][4], const float *bias, int kk,
                                           int t) {
  const Gelu16 g = gelu_bias16(f4(c[0]), f4(c[1]), f4(c[2]), f4(c[3]),
                               bias_pair(bias, 16 * kk + 2 * t), bias_pair(bias, 16 * kk + 8 + 2 * t),
                               bias_pair(bias, 16 * kk + 16 + 2 * t),
                               bias_pair(bias, 16 * kk + 24 + 2 * t));
  a0[0] = pack_bf16(g.v[0].x, g.v[0].y);
  a0[1] = pack_bf16(g.v[0].z, g.v[0].w);
  a0[2] = pack_bf16(g.v[1].x, g.v[1].y);
  a0[3] = pack_bf16(g.v[1].z, g.v[1].w);
  a1[0] = pack_bf16(g.v[2].x, g.v[2].y);
  a1[1] = pack_bf16(g.v[2].z, g.v[2].w);
  a1[2] = pack_bf16(g.v[3].x, g.v[3].y);
  a1[3] = pack_bf16(g.v[3].z, g.v[3].w);
}

// As gelu_pack2 for rows 0..7 only; rows 8..15 (not in use) become zero.
__device__ __forceinline__ void gelu_pack2_low(uint32_t (&a0)[4], uint32_t (&a1)[4],
                                               const float (&c)[4][4], const float *bias, int kk,
                                               int t) {
  const Gelu8 g = gelu_bias8(make_float4(c[0][0], c[0][1], c[1][0], c[1][1]),
                             make_float4(c[2][0], c[2][1], c[3][0], c[3][1]),
                             bias_pair(bias, 16 * kk + 2 * t), bias_pair(bias, 16 * kk + 8 + 2 * t),
                             bias_pair(bias, 16 * kk + 16 + 2 * t),
                             bias_pair(bias, 16 * kk + 24 + 2 * t));
  a0[0] = pack_bf16(g.lo.x, g.lo.y);
  a0[1] = 0u;
  a0[2] = pack_bf16(g.lo.z, g.lo.w);
  a0[3] = 0u;
  a1[0] = pack_bf16(g.hi.x, g.hi.y);
  a1[1] = 0u;
  a1[2] = pack_bf16(g.hi.z, g.hi.w);
  a1[3] = 0u;
}

// Dense layer of the node MLP: 16 rows, KT k-tiles of input fragments `in`,
// 128 outputs (8 pairs of n-tiles), bias + GELU into fragments `out`.
template <int KT>
__device__ __forceinline__ void node_layer(uint32_t (&out)[8][4], const uint32_t (&in)[KT][4],
                                           const bf16 *W, int ld, const float *bias, int lane,
                                           int t) {
#pragma unroll
  for (int kk = 0; kk < 8; kk += 2) {
    float c[4][4] = {};
#pragma unroll
    for (int q = 0; q < KT; ++q) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t bq[4];
        load_b2(bq, W, ld, 2 * (kk + h), q, lane);
        mma_bf16(c[2 * h], in[q], bq[0], bq[1]);
        mma_bf16(c[2 * h + 1], in[q], bq[2], bq[3]);
      }
    }
    gelu_pack2(out[kk], out[kk + 1], c, bias, kk, t);
  }
}

__global__ void __launch_bounds__(kFusedWarpsPerCta * 32, 1) sur_fused_kernel(const FusedArgs a) {
  constexpr unsigned FULL = 0xffffffffu;
  extern __shared__ __align__(16) unsigned char smem[];
  bf16 *sw = reinterpret_cast<bf16 *>(smem);
  float *sb = reinterpret_cast<float *>(smem + (size_t)kSmWeights * 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  bf16 *snode = reinterpret_cast<bf16 *>(smem + (size_t)kSmWeights * 2 + (size_t)kSmBias * 4) +
                warp * kSmWarp;
  bf16 *sedge = snode + 16 * kLdX;  // [kK][16][kLdX]
  unsigned char *s_agent = reinterpret_cast<unsigned char *>(sedge + kK * 16 * kLdX);  // [16]

  // stage the weights (32-bit words; every matrix offset and row length is even)
  {
    struct M { int dst, ld, src, rows, cols; };
    const M mats[5] = {{kSmE1, kLdE1, kOffWe1, 64, 16}, {kSmE2, kLdE2, kOffWe2, 64, 64},
                       {kSmN1, kLdN1, kOffW1, 128, 80}, {kSmN2, kLdN2, kOffW2, 128, 128},
                       {kSmN3, kLdN3, kOffW3, 8, 128}};
    for (int m = 0; m < 5; ++m) {
      const int wpr = mats[m].cols / 2;
      const uint32_t *src = reinterpret_cast<const uint32_t *>(a.w + mats[m].src);
      for (int q = threadIdx.x; q < mats[m].rows * wpr; q += blockDim.x) {
        const int r = q / wpr, c = q % wpr;
        reinterpret_cast<uint32_t *>(sw + mats[m].dst + r * mats[m].ld)[c] = src[r * wpr + c];
      }
    }
    for (int q = threadIdx.x; q < kSmBias; q += blockDim.x) {
      int src;
      if (q < 64) src = kOffbe1 + q;
      else if (q < 128) src = kOffbe2 + q - 64;
      else if (q < 256) src = kOffb1 + q - 128;
      else if (q < 384) src = kOffb2 + q - 256;
      else src = kOffb3 + q - 384;
      sb[q] = a.p[src];
    }
  }
  __syncthreads();
  const float *be1 = sb, *be2 = sb + 64, *bn1 = sb + 128, *bn2 = sb + 256, *bn3 = sb + 384;
  const bf16 *We1 = sw + kSmE1, *We2 = sw + kSmE2, *Wn1 = sw + kSmN1, *Wn2 = sw + kSmN2,
             *Wn3 = sw + kSmN3;
  const int g = lane >> 2, t = lane & 3;
  const int i = lane & 15;  // the agent this lane stands for (lanes 16..31 repeat 0..15)

  for (int e = blockIdx.x * kFusedWarpsPerCta + warp; e < a.E; e += gridDim.x * kFusedWarpsPerCta) {
    __syncwarp();  // the previous env's reads of this warp's feature rows are done
    const size_t b = (size_t)e * a.N;
    const float x = a.px[b + i], y = a.py[b + i], vx = a.vx[b + i], vy = a.vy[b + i];
    const float4 pr = a.param[b + i];
    const float r = pr.z, im = pr.x;
    const float *ac = a.actions + ((size_t)e * a.A + i) * 3;
    const float ax = ac[0], ay = ac[1];
    // the K nearest other agents within the radius (ties: lower index first)
    float bd[kK];
    int bj[kK];
#pragma unroll
    for (int k = 0; k < kK; ++k) {
      bd[k] = 0.f;
      bj[k] = i;
    }
    int n = 0;
    for (int j = 0; j < kAgents; ++j) {
      const float xj = __shfl_sync(FULL, x, j), yj = __shfl_sync(FULL, y, j);
      const float dx = xj - x, dy = yj - y;
      const float d = sqrtf(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)));
      if (j != i && d < kRadius && (n < kK || bd[kK - 1] > d)) {
        // insertion into the sorted list of the n kept (unrolled: registers)
        bool placed = false;
#pragma unroll
        for (int p = kK - 1; p >= 0; --p) {
          // slot p takes: the new one if it lands here, else its predecessor
          // if the new one lands before it, else keeps its own
          if (p <= n && !placed) {
            const bool before = p > 0 && bd[p - 1] > d;
            if (!before) {
              bd[p] = d;
              bj[p] = j;
              placed = true;
            } else {
              bd[p] = bd[p - 1];
              bj[p] = bj[p - 1];
            }
          }
        }
        if (n < kK) ++n;
      }
    }
    const int n_max = __reduce_max_sync(FULL, n);
    // Rows of every tile hold the agents sorted by neighbour count (most
    // first, ties by index): slot k is then in use exactly in its first c_k
    // rows, and a slot with c_k <= 8 skips the GELUs of rows 8..15.
    int row = 0;
    for (int j = 0; j < kAgents; ++j) {
      const int nj = __shfl_sync(FULL, n, j);
      row += (nj > n || (nj == n && j < i)) ? 1 : 0;
    }
    if (lane < 16) {
      s_agent[row] = (unsigned char)i;
      float nf[16];
      nf[0] = 10.f * vx;
      nf[1] = 10.f * vy;
      nf[2] = ax * im;
      nf[3] = ay * im;
      nf[4] = 10.f * r;
      nf[5] = im;
      nf[6] = fminf(1.f - x - r, kRadius) / kRadius;
      nf[7] = fminf(1.f + x - r, kRadius) / kRadius;
      nf[8] = fminf(1.f - y - r, kRadius) / kRadius;
      nf[9] = fminf(1.f + y - r, kRadius) / kRadius;
#pragma unroll
      for (int q = 10; q < 16; ++q) nf[q] = 0.f;
#pragma unroll
      for (int q = 0; q < 16; q += 2)
        *reinterpret_cast<uint32_t *>(snode + row * kLdX + q) = pack_bf16(nf[q], nf[q + 1]);
    }

    // edge features of every slot below n_max (lanes 0..15: slots 0..2,
    // lanes 16..31: slots 3..5, each for its agent i)
#pragma unroll
    for (int k = 0; k < kK; ++k) {
      const int jk = bj[k];
      const float xj = __shfl_sync(FULL, x, jk), yj = __shfl_sync(FULL, y, jk);
      const float vxj = __shfl_sync(FULL, vx, jk), vyj = __shfl_sync(FULL, vy, jk);
      const float rj = __shfl_sync(FULL, r, jk);
      if (k < n_max && (k / 3) == (lane >> 4)) {
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = 0.f;
        if (k < n) {
          v[0] = (xj - x) / kRadius;
          v[1] = (yj - y) / kRadius;
          v[2] = 10.f * (vxj - vx);
          v[3] = 10.f * (vyj - vy);
          v[4] = 10.f * rj;
          v[5] = (bd[k] - r - rj) / kRadius;
          v[6] = 1.f;
        }
        bf16 *dst = sedge + (k * 16 + row) * kLdX;
#pragma unroll
        for (int q = 0; q < 16; q += 2)
          *reinterpret_cast<uint32_t *>(dst + q) = pack_bf16(v[q], v[q + 1]);
      }
    }
    __syncwarp();

    // edge MLP over the neighbour slots, summed into M (rows g, g + 8)
    float Macc[8][4];
#pragma unroll
    for (int jt = 0; jt < 8; ++jt)
#pragma unroll
      for (int c = 0; c < 4; ++c) Macc[jt][c] = 0.f;
#pragma unroll 1
    for (int k = 0; k < n_max; ++k) {
      const int ck = __popc(__ballot_sync(FULL, n > k) & 0xffffu);  // rows in use
      const bool low_only = ck <= 8;                                 // warp-uniform
      uint32_t ae[4];
      load_a(ae, sedge + k * 16 * kLdX, kLdX, 0, lane);
      uint32_t he[4][4];
#pragma unroll
      for (int kk = 0; kk < 4; kk += 2) {
        float c[4][4] = {};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t bq[4];
          load_b2(bq, We1, kLdE1, 2 * (kk + h), 0, lane);
          mma_bf16(c[2 * h], ae, bq[0], bq[1]);
          mma_bf16(c[2 * h + 1], ae, bq[2], bq[3]);
        }
        if (low_only) gelu_pack2_low(he[kk], he[kk + 1], c, be1, kk, t);
        else gelu_pack2(he[kk], he[kk + 1], c, be1, kk, t);
      }
      const bool mg = g < ck, mg8 = g + 8 < ck;
#pragma unroll
      for (int jp = 0; jp < 4; jp += 2) {
        float c[4][4] = {};  // n-tiles 2 jp .. 2 jp + 3
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t bq[4];
            load_b2(bq, We2, kLdE2, 2 * (jp + h), kk, lane);
            mma_bf16(c[2 * h], he[kk], bq[0], bq[1]);
            mma_bf16(c[2 * h + 1], he[kk], bq[2], bq[3]);
          }
        }
        const float2 b0 = bias_pair(be2, 16 * jp + 2 * t), b1 = bias_pair(be2, 16 * jp + 8 + 2 * t);
        const float2 b2 = bias_pair(be2, 16 * jp + 16 + 2 * t);
        const float2 b3 = bias_pair(be2, 16 * jp + 24 + 2 * t);
        if (low_only) {
          const Gelu8 g = gelu_bias8(make_float4(c[0][0], c[0][1], c[1][0], c[1][1]),
                                     make_float4(c[2][0], c[2][1], c[3][0], c[3][1]), b0, b1, b2, b3);
          const float4 gv[2] = {g.lo, g.hi};
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            Macc[2 * (jp + h)][0] += mg ? gv[h].x : 0.f;
            Macc[2 * (jp + h)][1] += mg ? gv[h].y : 0.f;
            Macc[2 * (jp + h) + 1][0] += mg ? gv[h].z : 0.f;
            Macc[2 * (jp + h) + 1][1] += mg ? gv[h].w : 0.f;
          }
        } else {
          const Gelu16 g = gelu_bias16(f4(c[0]), f4(c[1]), f4(c[2]), f4(c[3]), b0, b1, b2, b3);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            Macc[2 * jp + i][0] += mg ? g.v[i].x : 0.f;
            Macc[2 * jp + i][1] += mg ? g.v[i].y : 0.f;
            Macc[2 * jp + i][2] += mg8 ? g.v[i].z : 0.f;
            Macc[2 * jp + i][3] += mg8 ? g.v[i].w : 0.f;
          }
        }
      }
    }

    // node MLP: z = [node features, bf(M)]
    uint32_t az[5][4];
    load_a(az[0], snode, kLdX, 0, lane);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      az[kk + 1][0] = pack_bf16(Macc[2 * kk][0], Macc[2 * kk][1]);
      az[kk + 1][1] = pack_bf16(Macc[2 * kk][2], Macc[2 * kk][3]);
      az[kk + 1][2] = pack_bf16(Macc[2 * kk + 1][0], Macc[2 * kk + 1][1]);
      az[kk + 1][3] = pack_bf16(Macc[2 * kk + 1][2], Macc[2 * kk + 1][3]);
    }
    uint32_t h1[8][4], h2[8][4];
    node_layer<5>(h1, az, Wn1, kLdN1, bn1, lane, t);
    node_layer<8>(h2, h1, Wn2, kLdN2, bn2, lane, t);
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      uint32_t bq[4];
      load_b1k2(bq, Wn3, kLdN3, q, lane);
      mma_bf16(o, h2[q], bq[0], bq[1]);
      mma_bf16(o, h2[q + 1], bq[2], bq[3]);
    }
    o[0] += bn3[2 * t];
    o[1] += bn3[2 * t + 1];
    o[2] += bn3[2 * t];
    o[3] += bn3[2 * t + 1];
    if (a.out) {
      float *o0 = a.out + ((size_t)e * kAgents + s_agent[g]) * 8 + 2 * t;
      float *o8 = a.out + ((size_t)e * kAgents + s_agent[g + 8]) * 8 + 2 * t;
      o0[0] = o[0];
      o0[1] = o[1];
      o8[0] = o[2];
      o8[1] = o[3];
    }
    if (!a.apply) continue;

    // agent i's outputs 0..3 (row `row`) sit in lanes 4 (row mod 8) (cols 0,
    // 1) and 4 (row mod 8) + 1 (cols 2, 3), components 0, 1 for rows < 8,
    // else 2, 3
    const int s0 = 4 * (row & 7), s1 = s0 + 1;
    const float q00 = __shfl_sync(FULL, o[0], s0), q01 = __shfl_sync(FULL, o[1], s0);
    const float q02 = __shfl_sync(FULL, o[2], s0), q03 = __shfl_sync(FULL, o[3], s0);
    const float q10 = __shfl_sync(FULL, o[0], s1), q11 = __shfl_sync(FULL, o[1], s1);
    const float q12 = __shfl_sync(FULL, o[2], s1), q13 = __shfl_sync(FULL, o[3], s1);
    const bool lo = row < 8;
    const float nx = fmaf(kXScale, lo ? q00 : q02, x);
    const float ny = fmaf(kXScale, lo ? q01 : q03, y);
    const float nvx = fmaf(kVScale, lo ? q10 : q12, vx);
    const float nvy = fmaf(kVScale, lo ? q11 : q13, vy);
    const bool finite = isfinite(nx) && isfinite(ny) && isfinite(nvx) && isfinite(nvy);
    float worst = wall_overlap(nx, ny, r);
    for (int j = 0; j < kAgents; ++j) {
      const float xj = __shfl_sync(FULL, nx, j), yj = __shfl_sync(FULL, ny, j);
      const float rj = __shfl_sync(FULL, r, j);
      const float dx = nx - xj, dy = ny - yj;
      if (j > i) worst = fmaxf(worst, r + rj - sqrtf(__fmaf_rn(dx, dx, __fmul_rn(dy, dy))));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) worst = fmaxf(worst, __shfl_xor_sync(FULL, worst, off));
    const bool fallback = !__all_sync(FULL, finite) || !(worst <= a.limit);
    if (fallback) {
      if (lane == 0) a.list[atomicAdd(a.list_len, 1)] = e;
    } else if (lane < 16) {
      a.px[b + i] = nx;
      a.py[b + i] = ny;
      a.vx[b + i] = nvx;
      a.vy[b + i] = nvy;
    }
  }
}

}  // namespace sur
}  // namespace vmas
