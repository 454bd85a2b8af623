// Learned surrogate of the world step (sm_103a): bfloat16 tensor-core GEMMs
// with FP32 accumulation (warp-level mma.sync m16n8k16 here, tcgen05 in
// gemm_tc.cuh), and the feature, aggregation, loss, GELU-backward and Adam
// kernels around them.
//
// Network (per node of a walled world: 16 agent spheres, and in the box
// world also 4 movable boxes; all widths fixed):
//   node features n (16), edge features e (16) for up to K = 6 nearest other
//   nodes within 0.3;  edge MLP he = bf(gelu(We1 bf(e) + be1)) (16 -> 64),
//   m = gelu(We2 he + be2) (64 -> 64), M = bf(sum of m over the edges);
//   node MLP z = [bf(n), M] (80), h1 = bf(gelu(W1 z + b1)) (-> 128),
//   h2 = bf(gelu(W2 h1 + b2)) (-> 128), out = W3 h2 + b3 (-> 8; 4 used by an
//   agent, 6 by a box);  next state x' = x + 0.01 out[0:2],
//   v' = v + 0.1 out[2:4], and for a box theta' = theta + 0.1 out[4],
//   omega' = omega + out[5].
// bf() rounds to bfloat16; gelu(z) = z (1 + erf(z / sqrt 2)) / 2.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "contact.cuh"

namespace vmas {
namespace sur {

constexpr int kK = 6;            // neighbour slots per node
constexpr int kAgents = 16;      // agents per env
constexpr int kEnts = 20;        // sphere world: 16 agents + 4 walls
constexpr int kBoxes = 4;        // box world: 16 agents + 4 boxes + 4 walls
constexpr int kNodesMax = kAgents + kBoxes;
constexpr float kRadius = 0.3f;
constexpr float kXScale = 0.01f, kVScale = 0.1f;
constexpr float kThScale = 0.1f, kOmScale = 1.0f;  // box angle and angular velocity

using bf16 = __nv_bfloat16;

// flat parameter layout (this order): We1 [64][16], be1 [64], We2 [64][64],
// be2 [64], W1 [128][80], b1 [128], W2 [128][128], b2 [128], W3 [8][128], b3 [8]
enum : int {
  kOffWe1 = 0, kOffbe1 = kOffWe1 + 64 * 16, kOffWe2 = kOffbe1 + 64, kOffbe2 = kOffWe2 + 64 * 64,
  kOffW1 = kOffbe2 + 64, kOffb1 = kOffW1 + 128 * 80, kOffW2 = kOffb1 + 128,
  kOffb2 = kOffW2 + 128 * 128, kOffW3 = kOffb2 + 128, kOffb3 = kOffW3 + 8 * 128,
  kParams = kOffb3 + 8
};

// 1 + erf(x) by the rational approximation of Abramowitz & Stegun,
// Handbook of Mathematical Functions, 7.1.26 (Hastings): for x >= 0,
// erf(x) = 1 - q(x), q = (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) e^{-x^2},
// t = 1 / (1 + p x), |error| <= 1.5e-7; erf is odd, so 1 + erf(x) = q(|x|)
// for x < 0 (no cancellation in the tail).  Fewer instructions than erff,
// and an error far below the bfloat16 rounding every GELU output meets.
__device__ __forceinline__ float one_plus_erf(float x) {
  const float ax = fabsf(x);
  const float t = __fdividef(1.f, fmaf(0.3275911f, ax, 1.f));
  float poly = fmaf(1.061405429f, t, -1.453152027f);
  poly = fmaf(poly, t, 1.421413741f);
  poly = fmaf(poly, t, -0.284496736f);
  poly = fmaf(poly, t, 0.254829592f);
  const float q = poly * t * __expf(-ax * ax);
  return x < 0.f ? q : 2.f - q;
}

// The forward GELU, gelu(z) = z (1 + erf(z / sqrt 2)) / 2, from the same
// approximation written for z: with a = |z| and x = a / sqrt 2,
// z (1 + erf(x)) / 2 = max(z, 0) - a q / 2, and
//   a q / 2 = a e^{-z^2 / 2} (t sum_i (a_i / 2) t^{i-1}),  t = 1 / (1 + (p / sqrt 2) a).
// Two forms with bitwise the same values: gelu2 on packed pairs (the
// two-wide FP32 add/mul/fma of sm_100 and later, each half rounded as its
// scalar operation), gelu on one value with the same operations in the same
// order (explicitly rounded, so never contracted differently).  The
// exponential and reciprocal are the hardware approximations.
constexpr float kGeluP = 0.3275911f * 0.70710678118654752f;
constexpr float kGeluC = -0.72134752044448170f;  // -log2(e) / 2: e^{-z^2/2} = 2^{C z^2}
constexpr float kGeluA1 = 0.254829592f * 0.5f, kGeluA2 = -0.284496736f * 0.5f,
                kGeluA3 = 1.421413741f * 0.5f, kGeluA4 = -1.453152027f * 0.5f,
                kGeluA5 = 1.061405429f * 0.5f;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 f2_splat(float v) { return make_float2(v, v); }

__device__ __forceinline__ float2 gelu2(float2 z) {
  const float2 a = make_float2(fabsf(z.x), fabsf(z.y));
  const float2 d = f2_fma(a, f2_splat(kGeluP), f2_splat(1.f));
  const float2 t = make_float2(rcp_approx(d.x), rcp_approx(d.y));
  const float2 w = f2_mul(f2_mul(z, f2_splat(kGeluC)), z);
  const float2 e = make_float2(ex2_approx(w.x), ex2_approx(w.y));
  float2 poly = f2_fma(f2_splat(kGeluA5), t, f2_splat(kGeluA4));
  poly = f2_fma(poly, t, f2_splat(kGeluA3));
  poly = f2_fma(poly, t, f2_splat(kGeluA2));
  poly = f2_fma(poly, t, f2_splat(kGeluA1));
  const float2 r = f2_mul(f2_mul(a, e), f2_mul(poly, t));
  return f2_sub(make_float2(fmaxf(z.x, 0.f), fmaxf(z.y, 0.f)), r);
}

__device__ __forceinline__ float gelu(float z) {
  const float a = fabsf(z);
  const float t = rcp_approx(__fmaf_rn(a, kGeluP, 1.f));
  const float e = ex2_approx(__fmul_rn(__fmul_rn(z, kGeluC), z));
  float poly = __fmaf_rn(kGeluA5, t, kGeluA4);
  poly = __fmaf_rn(poly, t, kGeluA3);
  poly = __fmaf_rn(poly, t, kGeluA2);
  poly = __fmaf_rn(poly, t, kGeluA1);
  const float r = __fmul_rn(__fmul_rn(a, e), __fmul_rn(poly, t));
  return __fsub_rn(fmaxf(z, 0.f), r);
}

// gelu'(z) = (1 + erf(z / sqrt 2)) / 2 + z phi(z).
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * one_plus_erf(z * 0.70710678118654752f) +
         z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

// --------------------------------------------------------------- GEMM
// C[m, n] = sum_k A(m, k) B(k, n);  A(m, k) = TA ? A[k lda + m] : A[m lda + k],
// B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].  Grid (ceil(M/64), ceil(N/64),
// splits); split z sums k in [z kchunk, (z+1) kchunk) and writes its partial
// to out_f32 + z M ldc_f.
struct GemmArgs {
  int M, N, K;
  const bf16 *A;
  int lda;
  const bf16 *B;
  int ldb;
  const float *bias;  // [N] or null (added by split 0 only)
  int act;            // 0: none, 1: gelu (applied to the bf16 output)
  float *out_f32;     // optional
  int ldc_f;
  bf16 *out_bf;       // optional
  int ldc_b;
  int kchunk;
};

constexpr int kBM = 64, kBN = 64, kBK = 32, kPad = 8;

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g) {
  __shared__ __align__(16) bf16 As[kBM][kBK + kPad];  // [m][k]
  __shared__ __align__(16) bf16 Bs[kBN][kBK + kPad];  // [n][k]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  const int kbeg = blockIdx.z * g.kchunk;
  const int kend = min(g.K, kbeg + g.kchunk);
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gi = lane >> 2, ti = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  const bf16 zero = __float2bfloat16_rn(0.f);
  // 16-byte loads of 8 consecutive elements where the operand allows them
  const bool vecA = ((reinterpret_cast<uintptr_t>(g.A) | (uintptr_t)g.lda * 2) & 15u) == 0;
  const bool vecB = ((reinterpret_cast<uintptr_t>(g.B) | (uintptr_t)g.ldb * 2) & 15u) == 0;
  // Stage a 64 x 32 tile T[r][kk] of an operand X whose element (r, k) is at
  // X[k ld + r] (KMAJOR = false) or X[r ld + k] (true), rows < R, k < kend.
  auto stage = [&](bf16 (*T)[kBK + kPad], const bf16 *X, int ld, int r0, int R, int k0, bool vec,
                   bool kmajor) {
    for (int q = tid; q < kBM * kBK / 8; q += 128) {
      // chunk of 8 along the contiguous dimension
      const int a = kmajor ? q / (kBK / 8) : q % (kBM / 8);  // row chunk / row
      const int b = kmajor ? q % (kBK / 8) : q / (kBM / 8);  // k chunk / k
      if (kmajor) {
        const int r = r0 + a, k = k0 + 8 * b;
        if (vec && r < R && k + 8 <= kend) {
          *reinterpret_cast<uint4 *>(&T[a][8 * b]) =
              *reinterpret_cast<const uint4 *>(X + (size_t)r * ld + k);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i)
            T[a][8 * b + i] = (r < R && k + i < kend) ? X[(size_t)r * ld + k + i] : zero;
        }
      } else {
        const int r = r0 + 8 * a, k = k0 + b;
        if (vec && r + 8 <= R && k < kend) {
          const uint4 v = *reinterpret_cast<const uint4 *>(X + (size_t)k * ld + r);
          const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
          for (int i = 0; i < 8; ++i) T[8 * a + i][b] = e[i];
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i)
            T[8 * a + i][b] = (r + i < R && k < kend) ? X[(size_t)k * ld + r + i] : zero;
        }
      }
    }
  };
  for (int k0 = kbeg; k0 < kend; k0 += kBK) {
    // stage the tiles (bounds-checked, zero filled)
    stage(As, g.A, g.lda, m0, g.M, k0, vecA, !TA);
    stage(Bs, g.B, g.ldb, n0, g.N, k0, vecB, TB);
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kBK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
      // fragment pairs are adjacent bfloat16 values: one 32-bit load each
      auto ld2 = [](const bf16 *q) { return *reinterpret_cast<const uint32_t *>(q); };
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const int r = wm + a * 16 + gi, c = ks + 2 * ti;
        af[a][0] = ld2(&As[r][c]);
        af[a][1] = ld2(&As[r + 8][c]);
        af[a][2] = ld2(&As[r][c + 8]);
        af[a][3] = ld2(&As[r + 8][c + 8]);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int n = wn + b * 8 + gi, c = ks + 2 * ti;
        bfr[b][0] = ld2(&Bs[n][c]);
        bfr[b][1] = ld2(&Bs[n][c + 8]);
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
              "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
              : "+f"(acc[a][b][0]), "+f"(acc[a][b][1]), "+f"(acc[a][b][2]), "+f"(acc[a][b][3])
              : "r"(af[a][0]), "r"(af[a][1]), "r"(af[a][2]), "r"(af[a][3]), "r"(bfr[b][0]),
                "r"(bfr[b][1]));
    }
    __syncthreads();
  }
  // epilogue
  float *of = g.out_f32 ? g.out_f32 + (size_t)blockIdx.z * g.M * g.ldc_f : nullptr;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int m = m0 + wm + a * 16 + gi + (c >= 2 ? 8 : 0);
        const int n = n0 + wn + b * 8 + 2 * ti + (c & 1);
        if (m >= g.M || n >= g.N) continue;
        float v = acc[a][b][c];
        if (g.bias && blockIdx.z == 0) v += g.bias[n];
        if (of) of[(size_t)m * g.ldc_f + n] = v;
        if (g.out_bf) g.out_bf[(size_t)m * g.ldc_b + n] = __float2bfloat16_rn(g.act ? gelu(v) : v);
      }
}

// Sum of `splits` partial [M][N] blocks (split-K reduction).
__global__ void sum_partials_kernel(float *__restrict__ out, const float *__restrict__ part,
                                    int splits, size_t MN) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= MN) return;
  float s = 0.f;
#pragma unroll 16
  for (int z = 0; z < splits; ++z) s += part[(size_t)z * MN + t];  // in split order
  out[t] = s;
}

// Partial column sums of a [M][N] FP32 matrix (bias gradients): block c
// sums rows [c chunk, (c+1) chunk) of column threadIdx.x in row order into
// part[c][n]; sum_partials_kernel finishes.
__global__ void col_sum_kernel(float *part, const float *x, int M, int N, int chunk) {
  const int n = threadIdx.x;
  if (n >= N) return;
  const size_t r0 = (size_t)blockIdx.x * chunk;
  const size_t r1 = min((size_t)M, r0 + chunk);
  float s = 0.f;
  for (size_t m = r0; m < r1; ++m) s += x[m * N + n];
  part[(size_t)blockIdx.x * N + n] = s;
}

// ------------------------------------------------------------ features
// One thread per node row r = e * nodes + i, reading a world's state planes
// (entity e * N + j; the nodes are entities 0 .. nodes-1: 16 agents, then in
// the box world the 4 boxes; the walls are the last 4 entities), per-entity
// parameters {1/m, 1/I, half size a, half size b}, kinds and actions
// [E][A][3] (node i takes row i).  Writes node [R][16], edge [K][R][16]
// (bfloat16; slot-major: row k R + r is node r's k-th neighbour) and mask
// [K][R].
//   node  0: 10 vx, 1: 10 vy, 2: fx / m, 3: fy / m, 4: 10 R (bounding radius:
//         a sphere's radius, a box's half diagonal), 5: 1 / m, 6..9: the
//         gaps to the walls at x = +1, -1, y = +1, -1 of the bounding circle,
//         min(gap, 0.3) / 0.3; boxes only: 10: 1, 11: cos theta,
//         12: sin theta, 13: 0.1 omega, 14: 0.01 torque / I
//   edge  0: dx / 0.3, 1: dy / 0.3 (d = x_j - x_i), 2: 10 dvx, 3: 10 dvy,
//         4: 10 R_j, 5: (|d| - R_i - R_j) / 0.3, 6: 1; neighbour a box:
//         7: 1, 8: cos theta_j, 9: sin theta_j, 10: 0.1 omega_j
// An agent of the sphere world, and an agent's edge to an agent, read the
// same values in both worlds.
struct FeatureArgs {
  int E, N, A, nodes;
  const float *px, *py, *vx, *vy, *th, *om;
  const float4 *param;
  const uint8_t *kind;
  const float *actions;
  bf16 *node, *edge;
  float *mask;
};

__device__ __forceinline__ float bounding_radius(const float4 pr, uint32_t kind) {
  return (kind & 3u) == 1u ? sqrtf(pr.z * pr.z + pr.w * pr.w) : pr.z;
}

// 16 floats as 16 bfloat16 (round to nearest even) in two 16-byte stores;
// dst is 32-byte aligned (a row of 16).
__device__ __forceinline__ void store_bf16x16(bf16 *dst, const float (&v)[16]) {
  uint32_t w[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);  // .x at the lower address
    w[q] = *reinterpret_cast<const uint32_t *>(&h);
  }
  uint4 *d4 = reinterpret_cast<uint4 *>(dst);
  d4[0] = make_uint4(w[0], w[1], w[2], w[3]);
  d4[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

__global__ void features_kernel(const FeatureArgs f) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int R = f.E * f.nodes;
  if (r >= R) return;
  const int e = r / f.nodes, i = r % f.nodes;
  const size_t b = (size_t)e * f.N;
  const float x = f.px[b + i], y = f.py[b + i], vx = f.vx[b + i], vy = f.vy[b + i];
  const float4 pi = f.param[b + i];
  const bool box_i = (f.kind[b + i] & 3u) == 1u;
  const float ri = bounding_radius(pi, f.kind[b + i]), im = pi.x;
  const float *a = f.actions + ((size_t)e * f.A + i) * 3;
  float nf[16];
  nf[0] = 10.f * vx;
  nf[1] = 10.f * vy;
  nf[2] = a[0] * im;
  nf[3] = a[1] * im;
  nf[4] = 10.f * ri;
  nf[5] = im;
  const float gaps[4] = {1.f - x - ri, 1.f + x - ri, 1.f - y - ri, 1.f + y - ri};
#pragma unroll
  for (int q = 0; q < 4; ++q) nf[6 + q] = fminf(gaps[q], kRadius) / kRadius;
#pragma unroll
  for (int q = 10; q < 16; ++q) nf[q] = 0.f;
  if (box_i) {
    const float th = f.th[b + i];
    nf[10] = 1.f;
    nf[11] = cosf(th);
    nf[12] = sinf(th);
    nf[13] = 0.1f * f.om[b + i];
    nf[14] = 0.01f * a[2] * pi.y;
  }
  store_bf16x16(f.node + (size_t)r * 16, nf);
  // the K nearest other nodes within the radius (ties: lower index first),
  // kept sorted in registers: +inf marks an empty place, and a new distance
  // goes after every kept one that is not larger (insertion, unrolled)
  float bd[kK];
  int bj[kK];
#pragma unroll
  for (int k = 0; k < kK; ++k) {
    bd[k] = __int_as_float(0x7f800000);
    bj[k] = 0;
  }
  for (int j = 0; j < f.nodes; ++j) {
    if (j == i) continue;
    const float dx = f.px[b + j] - x, dy = f.py[b + j] - y;
    const float d = sqrtf(__fmaf_rn(dx, dx, __fmul_rn(dy, dy)));
    if (!(d < kRadius)) continue;
#pragma unroll
    for (int q = kK - 1; q > 0; --q) {
      const bool mv = bd[q - 1] > d;          // the place below is larger: it moves up
      const bool put = !mv && bd[q] > d;      // d belongs here
      bj[q] = mv ? bj[q - 1] : (put ? j : bj[q]);
      bd[q] = mv ? bd[q - 1] : (put ? d : bd[q]);
    }
    if (bd[0] > d) {
      bd[0] = d;
      bj[0] = j;
    }
  }
  int n = 0;
#pragma unroll
  for (int k = 0; k < kK; ++k) n += bd[k] < kRadius ? 1 : 0;
#pragma unroll
  for (int k = 0; k < kK; ++k) {  // unrolled: bd and bj stay in registers
    const size_t row = (size_t)k * R + r;
    float v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = 0.f;
    float mk = 0.f;
    if (k < n) {
      const int j = bj[k];
      const uint32_t kj = f.kind[b + j];
      const float rj = bounding_radius(f.param[b + j], kj);
      v[0] = (f.px[b + j] - x) / kRadius;
      v[1] = (f.py[b + j] - y) / kRadius;
      v[2] = 10.f * (f.vx[b + j] - vx);
      v[3] = 10.f * (f.vy[b + j] - vy);
      v[4] = 10.f * rj;
      v[5] = (bd[k] - ri - rj) / kRadius;
      v[6] = 1.f;
      if ((kj & 3u) == 1u) {
        const float thj = f.th[b + j];
        v[7] = 1.f;
        v[8] = cosf(thj);
        v[9] = sinf(thj);
        v[10] = 0.1f * f.om[b + j];
      }
      mk = 1.f;
    }
    store_bf16x16(f.edge + row * 16, v);
    f.mask[row] = mk;
  }
}

// ---- Edge compaction --------------------------------------------------
// Of the K neighbour slots of a row only the first (its neighbour count)
// are in use, about 15 % of all slots on the paper-scale scenes.  The edge
// MLP runs on the slots in use only: an exclusive scan over the slot-major
// flags (mask[rk] != 0, rk = k R + r) gives each used slot its position pos[rk]
// (-1 for the others) in a compact edge array, kept in slot-major order.
// Three kernels: block scans, one scan of the block sums, then the compaction
// (positions made global, edge features gathered, emap[pos] = rk).
constexpr int kScanThreads = 256, kScanPer = 8;
constexpr int kScanBlock = kScanThreads * kScanPer;  // flags per block

__global__ void __launch_bounds__(kScanThreads) edge_scan_blocks_kernel(size_t n, const float *mask,
                                                                        int *pos, int *bsum) {
  __shared__ int s_w[kScanThreads / 32];
  const size_t b0 = (size_t)blockIdx.x * kScanBlock + (size_t)threadIdx.x * kScanPer;
  int f[kScanPer], cnt = 0;
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    f[u] = b0 + u < n && mask[b0 + u] != 0.f;
    cnt += f[u];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  int base = incl - cnt;
  for (int w = 0; w < warp; ++w) base += s_w[w];
#pragma unroll
  for (int u = 0; u < kScanPer; ++u) {
    if (b0 + u < n) pos[b0 + u] = f[u] ? base : -1;  // within the block
    base += f[u];
  }
  if (threadIdx.x == kScanThreads - 1) bsum[blockIdx.x] = base;  // the block's count
}

// Exclusive scan of the nb block counts in place (one block); total -> *total.
__global__ void __launch_bounds__(1024) edge_scan_sums_kernel(int nb, int *bsum, int *total) {
  __shared__ int s_w[32];
  const int per = (nb + 1023) / 1024;
  const int i0 = min(nb, (int)threadIdx.x * per), i1 = min(nb, i0 + per);
  int run = 0;
  for (int i = i0; i < i1; ++i) run += bsum[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  int base = incl - run;
  for (int w = 0; w < warp; ++w) base += s_w[w];
  for (int i = i0; i < i1; ++i) {
    const int v = bsum[i];
    bsum[i] = base;
    base += v;
  }
  if (threadIdx.x == 1023) *total = base;
}

// Global positions, and the used slots' features gathered in order.
__global__ void edge_compact_kernel(size_t n, int *pos, const int *bsum, const bf16 *edge,
                                    bf16 *edgec, int *emap) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || pos[i] < 0) return;
  const int q = pos[i] + bsum[i / kScanBlock];
  pos[i] = q;
  emap[q] = (int)i;
  const uint4 *src = reinterpret_cast<const uint4 *>(edge + i * 16);  // 16 bf16 = 2 x 16 B
  uint4 *dst = reinterpret_cast<uint4 *>(edgec + (size_t)q * 16);
  dst[0] = src[0];
  dst[1] = src[1];
}

// zin[r] = [node[r], bf(sum_k mask[k][r] gelu(ze2[pos[k][r]]))] (80 wide), the
// messages read from the compact edge array in slot order.  Four lanes per
// row (eight rows per warp): lane l of the row's group fetches the flags and
// positions of slots l and l + 4 (shared by width-4 shuffles), sums message
// columns 16l .. 16l + 15 (four 16-byte loads per slot in use), and lanes
// 0..1 copy the node features.
__global__ void __launch_bounds__(256) aggregate_compact_kernel(int R, const float *ze2c,
                                                                const float *mask, const int *pos,
                                                                const bf16 *node, bf16 *zin) {
  static_assert(kK <= 8, "slot flags are shared within 4 lanes, two each");
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t r = t >> 2;
  const int ql = threadIdx.x & 3;
  if ((t & ~(size_t)31) >> 2 >= (size_t)R) return;  // whole warps leave together
  const bool valid = r < (size_t)R;                  // later groups may have no row
  const float mk0 = valid && ql < kK ? mask[(size_t)ql * R + r] : 0.f;
  const int pk0 = valid && ql < kK && mk0 != 0.f ? pos[(size_t)ql * R + r] : 0;
  const float mk1 = valid && ql + 4 < kK ? mask[(size_t)(ql + 4) * R + r] : 0.f;
  const int pk1 = valid && ql + 4 < kK && mk1 != 0.f ? pos[(size_t)(ql + 4) * R + r] : 0;
  float sum[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) sum[q] = 0.f;
#pragma unroll
  for (int k = 0; k < kK; ++k) {
    const float m = __shfl_sync(0xffffffffu, k < 4 ? mk0 : mk1, k & 3, 4);
    const int q = __shfl_sync(0xffffffffu, k < 4 ? pk0 : pk1, k & 3, 4);
    if (m != 0.f) {
      const float4 *src = reinterpret_cast<const float4 *>(ze2c + (size_t)q * 64) + 4 * ql;
      float4 z[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) z[u] = src[u];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float2 g0 = gelu2(make_float2(z[u].x, z[u].y)), g1 = gelu2(make_float2(z[u].z, z[u].w));
        sum[4 * u] += m * g0.x;
        sum[4 * u + 1] += m * g0.y;
        sum[4 * u + 2] += m * g1.x;
        sum[4 * u + 3] += m * g1.y;
      }
    }
  }
  if (!valid) return;
  bf16 *out = zin + r * 80;
  if (ql < 2)
    reinterpret_cast<uint4 *>(out)[ql] = reinterpret_cast<const uint4 *>(node + r * 16)[ql];
  uint32_t w[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(sum[2 * i], sum[2 * i + 1]);
    w[i] = *reinterpret_cast<const uint32_t *>(&h);
  }
  uint4 *dst = reinterpret_cast<uint4 *>(out + 16) + 2 * ql;
  dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
  dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// Edge-message gradient on the compact array: d_ze2[e][c] =
// d_zin[r][16 + c] mask[rk] gelu'(ze2[e][c]), rk = emap[e], r = rk mod R,
// as bfloat16 (for the GEMMs), with the bias gradient's first column-sum
// stage fused in as in gelu_back_sum_kernel: block b takes edge rows
// [b chunk, (b + 1) chunk), thread c column c (blockDim.x >= 64), and writes
// the column's partial sum of the FP32 values to part[b][c].
__global__ void edge_back_sum_kernel(int R, int RE, const float *__restrict__ d_zin,
                                     const float *__restrict__ mask, const int *__restrict__ emap,
                                     const float *__restrict__ ze2c, bf16 *__restrict__ d_zbf,
                                     float *__restrict__ part, int chunk) {
  const int c = threadIdx.x;
  if (c >= 64) return;
  const size_t e0 = (size_t)blockIdx.x * chunk;
  const size_t e1 = min((size_t)RE, e0 + chunk);
  float s = 0.f;
#pragma unroll 8
  for (size_t e = e0; e < e1; ++e) {
    const size_t t = e * 64 + c;
    const size_t rk = (size_t)emap[e], r = rk % (size_t)R;
    const float v = d_zin[r * 80 + 16 + c] * mask[rk] * gelu_grad(ze2c[t]);
    d_zbf[t] = __float2bfloat16_rn(v);
    s += v;
  }
  part[(size_t)blockIdx.x * 64 + c] = s;
}

// d_z = d_h * gelu'(z) over [M][N] (N <= blockDim.x), with the bias
// gradient's first stage fused in: block b takes rows [b chunk, (b + 1)
// chunk), thread n column n, and writes the bfloat16 d_z (for the GEMMs) and
// the column's partial sum of the FP32 d_z to part[b][n], summed in row
// order as col_sum_kernel sums them (the FP32 d_z itself is not stored).
__global__ void gelu_back_sum_kernel(int M, int N, const float *__restrict__ d_h,
                                     const float *__restrict__ z, bf16 *__restrict__ d_zbf,
                                     float *__restrict__ part, int chunk) {
  const int n = threadIdx.x;
  if (n >= N) return;
  const size_t r0 = (size_t)blockIdx.x * chunk;
  const size_t r1 = min((size_t)M, r0 + chunk);
  float s = 0.f;
#pragma unroll 4
  for (size_t m = r0; m < r1; ++m) {
    const size_t t = m * N + n;
    const float v = d_h[t] * gelu_grad(z[t]);
    d_zbf[t] = __float2bfloat16_rn(v);
    s += v;
  }
  part[(size_t)blockIdx.x * N + n] = s;
}

// Loss: the mean of (out - y)^2 over the outputs each row uses (4 for an
// agent, 6 for a box: node i >= 16 of its env); y is [R][tw].  d_out =
// 2 (out - y) / count (unused columns zero), count = the used outputs of all
// rows; per-block partial sums of the squared error into part[blockIdx.x].
__global__ void loss_kernel(int R, int nodes, int tw, float count, const float *out, const float *y,
                            float *d_out32, bf16 *d_outbf, float *part) {
  __shared__ float red[256];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  float se = 0.f;
  if (t < R * 8) {
    const int r = t / 8, c = t % 8;
    const int used = (r % nodes) < kAgents ? 4 : 6;
    float d = 0.f;
    if (c < used) {
      const float diff = out[(size_t)r * 8 + c] - y[(size_t)r * tw + c];
      se = diff * diff;
      d = 2.f * diff / count;
    }
    d_out32[t] = d;
    d_outbf[t] = __float2bfloat16_rn(d);
  }
  red[threadIdx.x] = se;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// One block of 256 threads: strided partial sums, then a tree.
__global__ void finish_loss_kernel(const float *part, int n, float count, float *loss) {
  __shared__ float red[256];
  float s = 0.f;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += part[q];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / count;
}

// Adam on FP32 master parameters; weights (not biases) mirrored to bfloat16.
__global__ void adam_kernel(size_t n, float *p, const float *g, float *m, float *v, bf16 *pbf,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float gt = g[t];
  const float mt = b1 * m[t] + (1.f - b1) * gt;
  const float vt = b2 * v[t] + (1.f - b2) * gt * gt;
  m[t] = mt;
  v[t] = vt;
  const float upd = lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  const float np = p[t] - upd;
  p[t] = np;
  if (pbf) pbf[t] = __float2bfloat16_rn(np);
}

// Applies the prediction to a world's state planes for every env whose
// predicted agents overlap each other, or the walls at +-1, by at most
// `limit`; every other env is left unchanged and appended to `list` (the
// plain step then advances it).  One thread per env.
constexpr int kPbWarps = 8;  // envs per 256-thread block of the prediction checks

struct PredictArgs {
  int E, N;
  float *px, *py, *vx, *vy;
  const float4 *param;
  const float *out;  // [E * 16][8]
  float limit;
  int *list, *list_len;
};

// Overlap of agent (x, y, r) with the walls at x = +-1, y = +-1.
__device__ __forceinline__ float wall_overlap(float x, float y, float r) {
  return fmaxf(fmaxf(x + r - 1.f, r - 1.f - x), fmaxf(y + r - 1.f, r - 1.f - y));
}

// One warp per env: lane i < 16 predicts agent i and its wall overlap, the
// 120 agent pairs are spread over the lanes, and a warp max gives the
// deepest overlap (any order gives the same value).
__global__ void __launch_bounds__(256) predict_kernel(const PredictArgs a) {
  constexpr int NA = kAgents, kPairs = NA * (NA - 1) / 2;
  __shared__ float4 s_p[kPbWarps][NA];  // predicted x, y and the radius
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * kPbWarps + w;
  if (e >= a.E) return;  // whole warps leave together
  const size_t b = (size_t)e * a.N;
  float px = 0.f, py = 0.f, pvx = 0.f, pvy = 0.f;
  float worst = -1e30f;  // deepest predicted overlap
  bool fin = true;
  if (lane < NA) {
    const float *o = a.out + ((size_t)e * NA + lane) * 8;
    px = fmaf(kXScale, o[0], a.px[b + lane]);
    py = fmaf(kXScale, o[1], a.py[b + lane]);
    pvx = fmaf(kVScale, o[2], a.vx[b + lane]);
    pvy = fmaf(kVScale, o[3], a.vy[b + lane]);
    const float r = a.param[b + lane].z;
    fin = isfinite(px) && isfinite(py) && isfinite(pvx) && isfinite(pvy);
    worst = wall_overlap(px, py, r);
    s_p[w][lane] = make_float4(px, py, r, 0.f);
  }
  const bool finite = __all_sync(0xffffffffu, fin);
  __syncwarp();
  const float4 *P = s_p[w];
  for (int q0 = lane; q0 < kPairs; q0 += 32) {
    int q = q0, i = 0;
    while (q >= NA - 1 - i) {  // pair q of (i, j), i < j < 16, i-major
      q -= NA - 1 - i;
      ++i;
    }
    const int j = i + 1 + q;
    const float dx = P[i].x - P[j].x, dy = P[i].y - P[j].y;
    worst = fmaxf(worst, P[i].z + P[j].z - sqrtf(__fmaf_rn(dx, dx, __fmul_rn(dy, dy))));
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if (!finite || !(worst <= a.limit)) {
    if (lane == 0) a.list[atomicAdd(a.list_len, 1)] = e;
    return;
  }
  if (lane < NA) {
    a.px[b + lane] = px;
    a.py[b + lane] = py;
    a.vx[b + lane] = pvx;
    a.vy[b + lane] = pvy;
  }
}

// Box world: applies the prediction (agents x, y, vx, vy; boxes also theta,
// omega) to every env whose predicted bodies overlap one another, or the
// walls at +-1, by at most `limit` (sphere-sphere by centre distance,
// sphere-box and box-box by the step's own narrow phase, a box against a
// wall by its deepest corner); every other env is left unchanged and
// appended to `list`.
struct PredictBoxArgs {
  int E, N;
  float *px, *py, *vx, *vy, *th, *om;
  const float4 *param;
  const float *out;  // [E * 20][8]
  float limit;
  int *list, *list_len;
};

// One warp per env: lane i < 20 predicts node i (as the state it would
// write), the 210 overlap tests (16 agents against the walls, 120 agent
// pairs, 64 agent-box pairs, 4 boxes' corners against the walls, 6 box
// pairs) are spread over the lanes, and the deepest overlap is their
// maximum (any order gives the same value).  Over the limit, or any
// prediction not finite: the env is listed for the plain step; otherwise
// the lanes write the predicted state.
__global__ void __launch_bounds__(256) predict_box_kernel(const PredictBoxArgs a) {
  constexpr int NB = kNodesMax, NA = kAgents, NX = NB - NA;  // 20 nodes: 16 agents, 4 boxes
  constexpr int kWall = NA, kPair = kWall + NA * (NA - 1) / 2, kSB = kPair + NA * NX,
                kCorner = kSB + NX, kItems = kCorner + NX * (NX - 1) / 2;
  __shared__ float4 s_pose[kPbWarps][NB];  // predicted x, y, cos theta, sin theta
  __shared__ float2 s_half[kPbWarps][NB];  // radius (agents) or half sizes (boxes)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int e = blockIdx.x * kPbWarps + w;
  if (e >= a.E) return;  // whole warps leave together
  const size_t b = (size_t)e * a.N;
  float px = 0.f, py = 0.f, pvx = 0.f, pvy = 0.f, pth = 0.f, pom = 0.f;
  bool fin = true;
  if (lane < NB) {
    const float *o = a.out + ((size_t)e * NB + lane) * 8;
    px = fmaf(kXScale, o[0], a.px[b + lane]);
    py = fmaf(kXScale, o[1], a.py[b + lane]);
    pvx = fmaf(kVScale, o[2], a.vx[b + lane]);
    pvy = fmaf(kVScale, o[3], a.vy[b + lane]);
    pth = lane < NA ? a.th[b + lane] : fmaf(kThScale, o[4], a.th[b + lane]);
    pom = lane < NA ? a.om[b + lane] : fmaf(kOmScale, o[5], a.om[b + lane]);
    fin = isfinite(px) && isfinite(py) && isfinite(pvx) && isfinite(pvy) && isfinite(pth) &&
          isfinite(pom);
    const float4 pr = a.param[b + lane];
    const bool box = lane >= NA;
    s_pose[w][lane] = make_float4(px, py, box ? cosf(pth) : 1.f, box ? sinf(pth) : 0.f);
    s_half[w][lane] = make_float2(pr.z, pr.w);
  }
  const bool finite = __all_sync(0xffffffffu, fin);
  __syncwarp();
  float worst = -1e30f;  // deepest predicted overlap
  if (finite) {
    const float4 *P = s_pose[w];
    const float2 *H = s_half[w];
    for (int it = lane; it < kItems; it += 32) {
      if (it < kWall) {
        worst = fmaxf(worst, wall_overlap(P[it].x, P[it].y, H[it].x));
      } else if (it < kPair) {
        int q = it - kWall, i = 0;
        while (q >= NA - 1 - i) {  // pair q of (i, j), i < j < 16, i-major
          q -= NA - 1 - i;
          ++i;
        }
        const int j = i + 1 + q;
        const float dx = P[i].x - P[j].x, dy = P[i].y - P[j].y;
        worst = fmaxf(worst, H[i].x + H[j].x - sqrtf(__fmaf_rn(dx, dx, __fmul_rn(dy, dy))));
      } else if (it < kSB) {
        const int i = (it - kPair) / NX, j = NA + (it - kPair) % NX;
        Hit h;
        if (hit_sphere_box(P[i].x, P[i].y, H[i].x, P[j].x, P[j].y, P[j].z, P[j].w, H[j].x, H[j].y,
                           h))
          worst = fmaxf(worst, -h.g);
      } else if (it < kCorner) {
        const int i = NA + it - kSB;
        const float c = P[i].z, sn = P[i].w;
        for (int k = 0; k < 4; ++k) {  // corners against the walls
          const float u = (k == 1 || k == 2) ? H[i].x : -H[i].x, v = k >= 2 ? H[i].y : -H[i].y;
          const float cx = P[i].x + u * c - v * sn, cy = P[i].y + u * sn + v * c;
          worst = fmaxf(worst, fmaxf(fmaxf(cx - 1.f, -1.f - cx), fmaxf(cy - 1.f, -1.f - cy)));
        }
      } else {
        int q = it - kCorner, i = 0;
        while (q >= NX - 1 - i) {  // box pair q of (i, j), i < j < 4
          q -= NX - 1 - i;
          ++i;
        }
        const int bi = NA + i, bj = NA + i + 1 + q;
        const Poly A{P[bi].x, P[bi].y, P[bi].z, P[bi].w, H[bi].x, H[bi].y, true};
        const Poly B{P[bj].x, P[bj].y, P[bj].z, P[bj].w, H[bj].x, H[bj].y, true};
        Hit h;
        if (hit_poly_poly(A, B, h)) worst = fmaxf(worst, -h.g);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) worst = fmaxf(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if (!finite || !(worst <= a.limit)) {
    if (lane == 0) a.list[atomicAdd(a.list_len, 1)] = e;
    return;
  }
  if (lane < NB) {
    a.px[b + lane] = px;
    a.py[b + lane] = py;
    a.vx[b + lane] = pvx;
    a.vy[b + lane] = pvy;
    if (lane >= NA) {
      a.th[b + lane] = pth;
      a.om[b + lane] = pom;
    }
  }
}

// The nodes' (x, y, vx, vy, theta, omega) rows [E * nodes][6] of a world's
// planes.
__global__ void save_nodes_kernel(int E, int N, int nodes, const float *planes, size_t EN,
                                  float *save) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= E * nodes) return;
  const size_t g = (size_t)(r / nodes) * N + r % nodes;
#pragma unroll
  for (int f = 0; f < 6; ++f) save[(size_t)r * 6 + f] = planes[f * EN + g];
}

// Training targets [E * nodes][tw]: the step's deltas over (0.01, 0.01, 0.1,
// 0.1) and, when tw = 6, (0.1, 1) for theta and omega (0 for agents).
__global__ void targets_kernel(int E, int N, int nodes, int tw, const float *planes, size_t EN,
                               const float *save, float *target) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= E * nodes) return;
  const size_t g = (size_t)(r / nodes) * N + r % nodes;
  const float *s0 = save + (size_t)r * 6;
  float *t = target + (size_t)r * tw;
  const float sc[6] = {kXScale, kXScale, kVScale, kVScale, kThScale, kOmScale};
  for (int f = 0; f < tw; ++f)
    t[f] = (r % nodes) < kAgents && f >= 4 ? 0.f : (planes[f * EN + g] - s0[f]) / sc[f];
}

}  // namespace sur
}  // namespace vmas
