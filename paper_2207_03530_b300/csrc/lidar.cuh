// LIDAR ray casts (VMAS section 3: agents can carry LIDAR sensors), FP32.
//
// Every actuated entity casts n_rays rays from its centre at angles
// th + 2 pi k / n_rays; a ray reports the smallest distance t in
// [0, range] at which it meets another collidable entity (0 when its origin
// lies inside one), or `range` when it meets none.  Spheres are discs, boxes
// filled rectangles, lines segments (a ray exactly parallel to a segment
// misses it).  One CTA per environment: its collidable bodies are staged in
// shared memory grouped by shape, so that every loop tests one shape, and
// threads take (agent, ray) items, an agent's rays in consecutive lanes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "step.cuh"

namespace vmas {

struct LidarParams {
  int E, N, A, R;
  float range;
  const float *px, *py, *th;
  const float4 *param;  // {1/m, 1/I, ha, hb}
  const uint8_t *kind;
  float *out;           // [E][A][R]
};

// Entry distance of the ray o + t d (|d| = 1) into one body: 0 when o lies
// inside it, +inf on a miss.  Written without branches: a warp's lanes cast
// different rays at the same body, and every select costs less than a
// divergent early exit.
// Distances are absolute (at most the range), so the nearer root is taken
// as -b - sqrt(disc): its cancellation costs relative, not absolute, accuracy.
// Divides use the fast reciprocal (within 2 ulp) and the square root the
// hardware reciprocal square root (disc * rsqrt(disc)): both err by about
// 1e-7 of a unit-range distance.
__device__ __forceinline__ float ray_sphere(float ox, float oy, float dx, float dy, float4 b) {
  // b = {x, y, r, -}
  const float inf = __int_as_float(0x7f800000);
  const float px = ox - b.x, py = oy - b.y;
  const float cq = px * px + py * py - b.z * b.z;
  const float bb = px * dx + py * dy;
  const float disc = bb * bb - cq;
  const float t = -bb - (disc > 0.f ? disc * rsqrtf(disc) : 0.f);
  return cq <= 0.f ? 0.f : ((bb >= 0.f || disc < 0.f) ? inf : t);  // inside; away or past
}

// b = {x, y, cos, sin}, h = half sizes: slab test in the box frame.
__device__ __forceinline__ float ray_box(float ox, float oy, float dx, float dy, float4 b,
                                         float2 h) {
  const float inf = __int_as_float(0x7f800000);
  const float px = ox - b.x, py = oy - b.y;
  const float lx = b.z * px + b.w * py, ly = -b.w * px + b.z * py;
  const float ldx = b.z * dx + b.w * dy, ldy = -b.w * dx + b.z * dy;
  const float ix = __fdividef(1.f, ldx), iy = __fdividef(1.f, ldy);
  const float ax = (-h.x - lx) * ix, bx = (h.x - lx) * ix;
  const float ay = (-h.y - ly) * iy, by = (h.y - ly) * iy;
  // a ray parallel to a slab misses when it starts outside it, else that
  // slab does not bound t
  const float txa = ldx == 0.f ? -inf : fminf(ax, bx);
  const float txb = ldx == 0.f ? (fabsf(lx) > h.x ? -inf : inf) : fmaxf(ax, bx);
  const float tya = ldy == 0.f ? -inf : fminf(ay, by);
  const float tyb = ldy == 0.f ? (fabsf(ly) > h.y ? -inf : inf) : fmaxf(ay, by);
  const float tmin = fmaxf(txa, tya), tmax = fminf(txb, tyb);
  const bool inside = fabsf(lx) <= h.x && fabsf(ly) <= h.y;
  return inside ? 0.f : ((tmin > tmax || tmax < 0.f) ? inf : fmaxf(tmin, 0.f));
}

// b = {x, y, cos, sin}, half length hl; a ray exactly parallel misses.
__device__ __forceinline__ float ray_line(float ox, float oy, float dx, float dy, float4 b,
                                          float hl) {
  const float inf = __int_as_float(0x7f800000);
  const float px = ox - b.x, py = oy - b.y;
  const float lx = b.z * px + b.w * py, ly = -b.w * px + b.z * py;
  const float ldx = b.z * dx + b.w * dy, ldy = -b.w * dx + b.z * dy;
  const float t = __fdividef(-ly, ldy);
  return (ldy != 0.f && t >= 0.f && fabsf(lx + t * ldx) <= hl) ? t : inf;
}

// Bytes of dynamic shared memory per CTA for N entities.
__host__ __device__ inline int lidar_smem_bytes(int N) { return N * (16 + 8 + 1); }

__global__ void __launch_bounds__(128) lidar_kernel(const LidarParams p) {
  extern __shared__ __align__(16) unsigned char lsm[];
  float4 *s_pose = reinterpret_cast<float4 *>(lsm);            // [N] by list slot
  float2 *s_half = reinterpret_cast<float2 *>(s_pose + p.N);   // [N] by list slot
  uint8_t *s_kind = reinterpret_cast<uint8_t *>(s_half + p.N);  // [N] by entity
  __shared__ int s_ent[VMAS_LIDAR_MAX_ENTITIES];    // entity of each list slot
  __shared__ int s_slot[VMAS_LIDAR_MAX_ENTITIES];   // list slot of each entity (-1: none)
  __shared__ int s_agent[VMAS_LIDAR_MAX_ENTITIES];  // k-th actuated entity
  __shared__ int s_start[4];                        // list starts: spheres, boxes, lines, end
  __shared__ int s_nact;
  const int e = blockIdx.x;
  const size_t eb = (size_t)e * p.N;
  for (int i = threadIdx.x; i < p.N; i += blockDim.x) {
    s_kind[i] = p.kind[eb + i];
    s_slot[i] = -1;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // the collidable bodies, grouped by shape (each group in entity order),
    // and the casters, compacted with warp votes
    const int lane = threadIdx.x;
    const unsigned lt = (1u << lane) - 1u;
    int n = 0;
    for (int sh = 0; sh < 3; ++sh) {
      if (lane == 0) s_start[sh] = n;
      for (int c0 = 0; c0 < p.N; c0 += 32) {
        const int i = c0 + lane;
        const uint32_t kd = i < p.N ? s_kind[i] : 0u;
        const bool in = i < p.N && (kd & 3u) == (uint32_t)sh && (kd & kCollidable);
        const unsigned m = __ballot_sync(0xffffffffu, in);
        if (in) {
          s_ent[n + __popc(m & lt)] = i;
          s_slot[i] = n + __popc(m & lt);
        }
        n += __popc(m);
      }
    }
    int na = 0;
    for (int c0 = 0; c0 < p.N; c0 += 32) {
      const int i = c0 + lane;
      const bool act = i < p.N && (s_kind[i] & kActuated);
      const unsigned m = __ballot_sync(0xffffffffu, act);
      const int k = na + __popc(m & lt);
      if (act && k < p.A) s_agent[k] = i;
      na += __popc(m);
    }
    if (lane == 0) {
      s_start[3] = n;
      s_nact = na < p.A ? na : p.A;
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < s_start[3]; q += blockDim.x) {
    const int i = s_ent[q];
    const float4 pr = p.param[eb + i];
    float c = 1.f, s = 0.f;
    if ((s_kind[i] & 3u) != kSphere) body_axes(p.th[eb + i], c, s);
    const bool sphere = (s_kind[i] & 3u) == kSphere;
    // a sphere's slot holds {x, y, r, -}: one load per test
    s_pose[q] = make_float4(p.px[eb + i], p.py[eb + i], sphere ? pr.z : c, sphere ? 0.f : s);
    s_half[q] = make_float2(pr.z, pr.w);
  }
  __syncthreads();
  const int nact = s_nact, b0 = s_start[1], l0 = s_start[2], end = s_start[3];
  const float inf = __int_as_float(0x7f800000);
  const float step = 6.283185307179586f / (float)p.R;
  for (int it = threadIdx.x; it < p.A * p.R; it += blockDim.x) {
    const int k = it / p.R, r = it - k * p.R;
    float best = p.range;
    if (k < nact) {
      const int i = s_agent[k];
      const int self = s_slot[i];  // the caster's own slot is skipped
      const float ox = p.px[eb + i], oy = p.py[eb + i];
      float dx, dy;
      body_axes(p.th[eb + i] + step * (float)r, dx, dy);
#pragma unroll 4
      for (int q = 0; q < b0; ++q) {
        const float4 b = s_pose[q];
        const float t = ray_sphere(ox, oy, dx, dy, b);
        best = fminf(best, q == self ? inf : t);
      }
#pragma unroll 2
      for (int q = b0; q < l0; ++q) {
        const float t = ray_box(ox, oy, dx, dy, s_pose[q], s_half[q]);
        best = fminf(best, q == self ? inf : t);
      }
#pragma unroll 2
      for (int q = l0; q < end; ++q) {
        const float t = ray_line(ox, oy, dx, dy, s_pose[q], s_half[q].x);
        best = fminf(best, q == self ? inf : t);
      }
    }
    p.out[((size_t)e * p.A + k) * p.R + r] = best;
  }
}

}  // namespace vmas
